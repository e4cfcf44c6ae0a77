/*
 * wilson_mg.h -- C-ABI of a GB300 (sm_103a) adaptive multigrid solver for the
 * lattice Wilson-Dirac equation D(U) psi = b (Babich et al., "Adaptive
 * multigrid algorithm for the lattice Wilson-Dirac operator", arXiv:1005.3043).
 *
 * Every numerical step runs in CUDA kernels of this library.  Plain pointers
 * and sizes only; no C++ or framework types cross this boundary.
 *
 * ---------------------------------------------------------------------------
 * Layouts at the boundary (all host- and device-pointer arguments)
 *   site index    s = x + L0*(y + L1*(z + L2*t)), mu = 0..3 is x, y, z, t
 *   complex       two doubles (re, im)
 *   links U       [mu 4][site][row 3][col 3] complex double
 *   fine spinor   [site][spin 4][colour 3] complex double, DeGrand-Rossi
 *                 (chiral) gamma basis: gamma5 = diag(1, 1, -1, -1)
 *   null vectors  [i < Nv][site][spin][colour] complex double
 *   coarse vector [X][2 Nv] complex double, X lexicographic over the coarse
 *                 lattice L/B; dof a = s*Nv + i with chirality s = 0 (spins
 *                 0,1) or 1 (spins 2,3)
 *   coarse op     [X][d 9][a][b] complex double, (D_c y)[X] = sum_d A[X][d] y[X+d],
 *                 d = 0 on-site, 1+2mu for X+mu, 2+2mu for X-mu
 * Boundary conditions: periodic in x, y, z; antiperiodic in t when
 * t_antiperiodic != 0.
 *
 * Ownership: the caller owns every buffer it passes; the library copies what
 * it keeps.  The context owns all device memory it allocates and frees it in
 * mg_destroy.  All work is issued on the stream given to mg_create; calls
 * taking host buffers synchronise that stream before returning.
 *
 * Errors: every int-returning call returns MG_OK (0) or a negative
 * mg_status; mg_last_error() gives a message.  A context is not thread-safe.
 * ---------------------------------------------------------------------------
 */
#ifndef WILSON_MG_H
#define WILSON_MG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_ctx mg_ctx;

enum mg_status {
    MG_OK = 0,
    MG_ERR_INVALID_ARG = -1,   /* bad size, null pointer, L not divisible by B */
    MG_ERR_NOT_SETUP = -2,     /* links / null vectors / coarse operator missing */
    MG_ERR_OOM = -3,           /* device allocation failed */
    MG_ERR_NOT_CONVERGED = -4, /* x holds the last iterate, info is filled */
    MG_ERR_NUMERIC = -5,       /* NaN/Inf, breakdown, rank-deficient block QR */
    MG_ERR_TIMEOUT = -6,       /* a bounded device wait gave up */
    MG_ERR_CUDA = -7           /* a CUDA runtime call failed */
};

/* Inner precision of the preconditioner and Krylov basis (the solution and
 * the true residual are always FP64).  MG_FP16: FP32 arithmetic with FP16
 * storage of the coarse operator of the CGNR coarse solve (one scale per
 * (aggregate, direction) block; needs an even nvec), of the links of the
 * smoother's Wilson operator (no scale: |U_ij| <= 1) and of the smoother's
 * residual and D-residual spinors (one FP32 scale per site, the site's
 * largest |re|, |im|) as selected by mg_params.smoother_fp16; the Krylov
 * basis, restriction and prolongation stay FP32. */
enum mg_precision { MG_FP64 = 0, MG_FP32 = 1, MG_FP16 = 2 };

/* Solver parameters (paper, Sec. III-IV; defaults from mg_default_params). */
typedef struct {
    int block[4];          /* aggregate (block) extent per direction, default 4^4 (Sec. III) */
    int nvec;              /* N_v near-null vectors; 2 N_v coarse dof per site */
    int setup_init_relax;  /* relaxation steps on each random vector (Sec. IV: 10) */
    int setup_iters;       /* truncated-MG iterations per group (Sec. IV: 5) */
    int setup_group;       /* prototypes refined together (Sec. IV: groups of 4) */
    int smoother_steps;    /* post-smoothing steps, V(0,n) cycle (Sec. IV: 4) */
    double omega;          /* smoother under-relaxation (Sec. III: 0.9) */
    int gcr_restart;       /* flexible GCR restart length (Sec. III: GCR(8); default 16) */
    double tol;            /* outer true relative residual ||b-Dx||/||b|| */
    double coarse_tol;     /* coarse CG-on-normal-equations relative residual (Sec. IV: 1e-3) */
    int max_outer;         /* maximum outer iterations (preconditioner applications) */
    int max_coarse;        /* maximum coarse iterations per cycle */
    double delta;          /* mixed precision: restart when ||r|| < delta * ||r at restart|| (0: off) */
    int prec_inner;        /* MG_FP64, MG_FP32 or MG_FP16: smoother, dslash, transfers, coarse solve, Krylov basis */
    int coarse_check;      /* coarse iterations between convergence checks read by the host */
    int coarse_kernel;     /* FP32/FP16 coarse solve: 0 (default) operator held on chip for the
                              whole solve, in tensor memory when each SM's share fits (FP16: its
                              products on the tensor cores when each SM holds at most 140 rows),
                              else in shared memory, else as 1; 1 operator read from global
                              memory into registers every iteration; 2 operator streamed through
                              a shared-memory ring (tests); 3 shared memory only (tests); 4 tensor
                              memory with the products on the CUDA cores (tests) */
    int smoother;          /* post-smoother: 0 (default) smoother_steps MR steps, each scaled by omega;
                              1 one GMRES(smoother_steps) application scaled by omega (Sec. III-IV:
                              GMRES(4)), smoother_steps <= 16, FP32/FP64 storage */
    int smoother_fp16;     /* MG_FP16 only, storage of the smoother's spinors and links (MR) or of its
                              Arnoldi basis (GMRES): 0 (default) FP16 when the FP32 working set
                              (MR: links + 3 spinors, 576 B per site; GMRES: k + 1 spinors, 96 B
                              each) exceeds the device L2, else FP32; 1 always FP16; 2 never */
    int coarse_form;       /* iteration form of the on-chip coarse solve (coarse_kernel 0, 2, 3, 4):
                              0 (default) Chronopoulos-Gear form, one grid-wide exchange per
                              iteration, the vectors other SMs read carrying epoch tags instead
                              of barriers; 1 textbook CGLS, two grid-wide exchanges per
                              iteration.  Same iterates in exact arithmetic */
    /* third level (Sec. IV: 3-level V(0,4) cycle with GMRES(4) post-relaxation on
       each level and a W-cycle); levels = 2 ignores the rest */
    int levels;            /* 2 (default) or 3 */
    int block2[4];         /* level-2 aggregates on the level-1 lattice (default 2^4; Sec. IV's
                              footnote: 2^3 x 4 on 24^3 x 64) */
    int nvec2;             /* N_v of level 2 (default 32), 2 nvec2 dof per level-2 site */
    int smoother_steps1;   /* level-1 post-smoothing: one GMRES(smoother_steps1) scaled by omega */
    int cycles1;           /* level-1 V-cycles per fine-grid correction (Sec. IV: 2, the W-cycle) */
} mg_params;

/* Outcome of one solve (Sec. IV reports outer iterations and fine matvecs). */
typedef struct {
    int outer_iters;       /* preconditioner applications (the paper's outer GCR count, Table I) */
    int coarse_iters;      /* total coarse-solver iterations */
    int fine_matvecs;      /* fine D applications, all precisions (the work unit of Fig. 1) */
    int restarts;          /* true-residual recomputations */
    double true_rel_res;   /* ||b - D x|| / ||b|| in FP64 */
    double solve_ms;       /* device time of the solve (CUDA events) */
    int status;
    double setup_ms;       /* device time of the context's last adaptive setup (0: none) */
    double dslash_bytes;   /* algorithmic bytes of the fine D applications of this solve: per
                              application and site the links, one input and one output spinor
                              in that application's storage (FP64 960, FP32 480, FP16 248 B) */
} mg_solve_info;

/* Fill p with the defaults (Sec. III-IV parameters where the paper gives them):
 * block 4^4, nvec 8, relax 10, iters 3, group 4,
 * smoother 4, omega 0.9, restart 16, tol 1e-10, coarse_tol 1e-3,
 * max_outer 1000, max_coarse 5000, delta 0, FP64, coarse_check 16, coarse_kernel 0,
 * smoother 0 (MR), smoother_fp16 0, coarse_form 0, levels 2, block2 2^4,
 * nvec2 32, smoother_steps1 4, cycles1 2. */
int mg_default_params(mg_params* p);

/* Create a context for the Wilson-Dirac system D(U) psi = b (eqs. 1-2) on an
 * L0 x L1 x L2 x L3 lattice.  dims[mu] must be a multiple of p->block[mu]
 * (geometric 4^4 aggregates, Sec. III).  stream is a cudaStream_t (NULL:
 * legacy default); the device current at this call owns the context.
 * Allocates the device buffers of the fine level; the coarse level is
 * allocated by mg_set_null_vectors / mg_setup.  *out is NULL on error. */
int mg_create(const int dims[4], int t_antiperiodic, const mg_params* p, void* stream, mg_ctx** out);

/* Free every device buffer of the context (synchronises its stream first).
 * Accepts NULL. */
void mg_destroy(mg_ctx* ctx);

/* Copy the SU(3) links U_x^mu of eq. 2 (host, boundary layout, 4*V*9
 * complex) to the device.  Synchronous.  Invalidates the coarse level (D_c
 * depends on U): run mg_setup or mg_set_null_vectors again. */
int mg_set_links(mg_ctx* ctx, const double* U);

/* As mg_set_links with U_dev in device memory (boundary layout, FP64, owned by
 * the caller).  Stream-ordered, no host synchronisation: the conversion waits
 * for the work already queued on `stream` (a cudaStream_t; NULL: legacy
 * default) and later work on `stream` waits for the conversion, so the caller
 * may overwrite or free U_dev after queuing it there. */
int mg_set_links_device(mg_ctx* ctx, const double* U_dev, void* stream);

/* Bare mass m of eq. (2).  After a setup the coarse operator is shifted in
 * place: D_c(m) = D_c(m0) + (m - m0) I, exact because P^dag P = I (eq. 4). */
int mg_set_mass(mg_ctx* ctx, double m);

/* Replace the solver parameters (Sec. III-IV) that do not change buffer sizes
 * (tolerances, smoother, restart <= the value at create, precision, ...);
 * nvec and block are fixed at create (MG_ERR_INVALID_ARG otherwise). */
int mg_set_params(mg_ctx* ctx, const mg_params* p);

/* Adaptive setup (Sec. II alpha-SA loop in the two-step form of Sec. IV) from
 * caller-provided random starts V0 (host, Nv fine vectors): relaxation, group
 * refinement with the truncated two-level method, block orthonormalisation
 * (eq. 4) and the Galerkin coarse operator D_c = P^dag D P.  The starts are
 * an argument, not a seed, so that any generator (and the CPU checker of the
 * tests) can supply identical vectors; the paper only asks for random ones.
 * Run at the lightest mass of interest (Sec. IV: the prototypes serve every
 * heavier mass); info.setup_ms of later solves reports its device time. */
int mg_setup(mg_ctx* ctx, const double* V0);

/* As mg_setup (Sec. II, IV) with the random starts in device memory
 * (boundary layout, FP64, owned by the caller; read before the call returns). */
int mg_setup_device(mg_ctx* ctx, const double* V0_dev);

/* Use the given prototypes (host, nv == p->nvec fine vectors) as they are:
 * block-orthonormalise them (eq. 4) and build D_c = P^dag D P (Sec. III).
 * MG_ERR_NUMERIC when an aggregate's prototypes are rank-deficient. */
int mg_set_null_vectors(mg_ctx* ctx, const double* V, int nv);

/* Read back the block-orthonormal prolongator columns of eq. 4 (host, Nv
 * fine vectors: column (X, s, i) is vector i on the sites of X and spins of
 * s, chirality kept as in Sec. III). */
int mg_get_prolongator(mg_ctx* ctx, double* P);

/* ---- the third level (levels = 3) -----------------------------------------
 * Level-1 vectors are coarse vectors (boundary coarse-vector layout [X1][2 Nv]).
 * Sec. III recurses the coarsening with the chiral components kept separate:
 * level-2 aggregates are block2 level-1 sites, level-2 dof (s, i) of chirality s.
 * Level-2 vectors [X2][2 nvec2], X2 lexicographic over the level-2 lattice
 * (level-1 extents / block2); the level-2 operator [X2][d 9][a][b] as D_c. */

/* Adaptive setup of level 2 (the two-step setup of Sec. IV applied to D_c:
 * setup_init_relax relaxation steps -- GMRES(1) applications, each equal to
 * one MR step -- on D_c v = 0 from each start, then groups of setup_group
 * prototypes refined by setup_iters iterations of the truncated two-level
 * method of levels 1 and 2), then P2 = block-orthonormalised prototypes and
 * A2 = P2^dag D_c P2.  V2: host, nvec2 random level-1 vectors.  Needs the
 * level-1 setup (mg_setup or mg_set_null_vectors) first; runs at the current
 * mass.  MG_ERR_NUMERIC on rank-deficient level-2 aggregates. */
int mg_setup_level2(mg_ctx* ctx, const double* V2);

/* Use the given level-1 vectors (host, nvec2) as level-2 prototypes as they
 * are: block-orthonormalise them and build A2 = P2^dag D_c P2 (Sec. III). */
int mg_set_level2_vectors(mg_ctx* ctx, const double* V2);

/* Read back the level-2 prolongator as nvec2 level-1 vectors (column (X2, s, i)
 * is vector i on the level-1 sites of X2 and dof of chirality s) and the
 * level-2 operator in FP64 (host). */
int mg_get_level2_prolongator(mg_ctx* ctx, double* P2);
int mg_get_level2_op(mg_ctx* ctx, double* A2);

/* e1 = the three-level method's coarse-grid correction of a level-1 residual
 * r1 (Sec. IV): cycles1 level-1 V-cycles on D_c e1 = r1 from e1 = 0, each
 * r2 = P2^dag r, level-2 CGNR to coarse_tol, e = P2 y2, one GMRES(smoother_
 * steps1) post-smoothing on D_c.  r1, e1: host level-1 vectors; prec as the
 * solve's inner precision. */
int mg_kcycle(mg_ctx* ctx, const double* r1, double* e1, int prec);

/* ---- the learned setup ------------------------------------------------------
 * The paper has no network: this one stands in for the random-start
 * relaxation that begins the Sec. IV setup (10 relaxation steps on each random
 * vector, a polynomial in the hopping term of eq. 2).  A gauge-covariant
 * parallel-transport convolution: four linear layers with 1, 8, 8, 8, 1
 * channels, out[a](x) = sum_b sum_d W[a][b][d] (T_d in[b])(x) over the site
 * (d = 0) and its eight neighbours (d = 1 + 2 mu: x + mu, 2 + 2 mu: x - mu),
 * (T_{+mu} p)(x) = U_mu(x) p(x + mu), (T_{-mu} p)(x) = U_mu(x - mu)^dag
 * p(x - mu), the antiperiodic sign across the t boundary, W[a][b][d] a 4x4
 * complex spin matrix.  Weights: 20736 complex doubles, the layers in order,
 * each [Cout][Cin][d 9][s 4][t 4] (out_s += W_st in_t).  Inputs eta: host
 * random fine spinors (boundary layout); the outputs are its prototypes.
 * Training target: the block projector P P^dag of the context's current level
 * (the plain setup's, eq. 4); loss |(1 - P P^dag) v|^2 / |v|^2 averaged over
 * the starts; gradient the Wirtinger 2 dLoss/d conj(W) in the weights' layout.
 * FP32 kernels, FP64 gradient sums and weights. */
int mg_nn_set_weights(mg_ctx* ctx, const double* W, int ncomplex);
int mg_nn_get_weights(mg_ctx* ctx, double* W, int ncomplex);
/* v_i = network(eta_i), i < n (host fine spinors). */
int mg_nn_forward(mg_ctx* ctx, const double* eta, double* v, int n);
/* loss (and, with grad != NULL, its gradient) over n starts; needs a level. */
int mg_nn_loss_grad(mg_ctx* ctx, const double* eta, int n, double* loss, double* grad);
/* steps Adam steps (learning rate lr, betas 0.9 / 0.999) on the current links
 * and level, each over the n starts; the mean loss of the first and of the
 * last step (each before its update) in *loss_first, *loss_last (may be NULL). */
int mg_nn_train(mg_ctx* ctx, const double* eta, int n, int steps, double lr, double* loss_first, double* loss_last);
/* The learned setup: prototypes v_i = network(eta_i), i < nvec, normalised,
 * in place of the random starts of the Sec. IV setup; then, as in mg_setup,
 * params.setup_init_relax relaxation steps (0 skips them) and the group
 * refinement, here with refine_iters truncated-cycle iterations per prototype
 * (0 skips it), then P and D_c (eq. 4, Sec. III).  info.setup_ms of later
 * solves reports its device time. */
int mg_setup_learned(mg_ctx* ctx, const double* eta, int refine_iters);

/* Read back the current prototypes V (the near-null vectors of Sec. II;
 * host, Nv fine vectors). */
int mg_get_null_vectors(mg_ctx* ctx, double* V);

/* Read back the Galerkin coarse operator D_c = P^dag D P (Sec. III, nearest
 * neighbour with 2Nv x 2Nv links) in FP64 (host, boundary coarse-operator
 * layout). */
int mg_get_coarse_op(mg_ctx* ctx, double* A);

/* Solve D x = b by MG-preconditioned flexible GCR (Sec. III), x0 = 0.
 * b, x: host fine spinors (FP64).  Returns MG_ERR_NOT_CONVERGED with x the
 * last iterate when max_outer is reached. */
int mg_solve(mg_ctx* ctx, const double* b, double* x, mg_solve_info* info);

/* As mg_solve (Sec. III) with b and x in device memory (boundary layout,
 * FP64, owned by the caller); synchronises the context stream. */
int mg_solve_device(mg_ctx* ctx, const double* b_dev, double* x_dev, mg_solve_info* info);

/* Solve D x_n = b_n (eq. 1) for nrhs sources together (12 spin-colour point
 * sources plus Gaussian sources, say; the paper solves one point source at a
 * time, Sec. IV): flexible GCR (Sec. III) in lockstep over the sources, each
 * with its own Krylov space and scalars, the fine-level steps per source and
 * the coarse solve of all sources as one batched CGNR on an RHS panel, its
 * stencil a dense contraction on the tensor cores (FP16 operator, FP16 hi+lo
 * panel, FP32 accumulation), its iterations replayed from a captured CUDA
 * graph.  b, x: nrhs consecutive host fine spinors; info: nrhs entries.
 * Needs prec_inner MG_FP32 or MG_FP16 (the smoother then follows the FP16
 * storage rules of mg_params.smoother_fp16) and 2*nvec a multiple of 16
 * (<= 128), nrhs <= 256; with MG_FP64 the sources are solved one after
 * another. */
int mg_solve_batched(mg_ctx* ctx, const double* b, double* x, int nrhs, mg_solve_info* info);

/* As mg_solve_batched with b and x in device memory (boundary layout, nrhs
 * consecutive fine spinors, owned by the caller). */
int mg_solve_batched_device(mg_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, mg_solve_info* info);

/* Red-black (even-odd) preconditioned CG, the solver Sec. IV compares MG-GCR
 * against (Fig. 1: Wilson matrix-vector products, Fig. 2: flops): CG on the
 * normal equations of the even-site Schur complement
 * Dhat = (4+m) - H_eo H_oe / (4+m) of eq. 2 (D = (4+m) - H), the odd sites
 * reconstructed as x_o = (b_o + H_oe x_e) / (4+m).  prec MG_FP32: the CG
 * iterates in FP32; each time its own residual has fallen by a factor 10 the
 * solution is accumulated in FP64, the residual recomputed in FP64 and the
 * CG continued from it with its search direction kept (reliable update);
 * MG_FP64: FP64 throughout.  Stops when ||b - D x|| <= tol ||b|| in
 * FP64 or after maxit CG iterations (MG_ERR_NOT_CONVERGED, x the last
 * iterate).  Needs even lattice extents.  Uses the context's links and mass,
 * no setup.  info: outer_iters = CG iterations, restarts = defect-correction
 * cycles, coarse_iters = 0, fine_matvecs = matrix products: one per Dhat or
 * Dhat^dag (two half-lattice hops each) and, per cycle, one each for the
 * right-hand side Dhat x_e = b_e + H_eo b_o / (4+m), the odd-site
 * reconstruction and the FP64 residual; dslash_bytes counts every half-lattice
 * hop (all 4V links, input and output half vectors).  b, x: host spinors. */
int mg_solve_eo_cg(mg_ctx* ctx, const double* b, double* x, double tol, int maxit, int prec, mg_solve_info* info);

/* As mg_solve_eo_cg with b and x in device memory (boundary layout, FP64,
 * owned by the caller); synchronises the context stream. */
int mg_solve_eo_cg_device(mg_ctx* ctx, const double* b_dev, double* x_dev, double tol, int maxit, int prec,
                          mg_solve_info* info);

/* Timing of the tensor-core batched coarse stencil (measurement hook, no
 * counterpart in the paper): `reps` launches of y = D_c x on a device panel of
 * nrhs columns (the chunk width from the autotuner), CUDA events on the
 * context stream; *ms_per_launch, and per launch the algorithmic bytes (the
 * FP16 embedded operator once, the FP32 panel read and written once) and the
 * useful flops (8 per complex multiply-add of D_c x_n).  Allocates and frees
 * two panels.  Same shape limits as mg_apply_coarse_batched with impl 0. */
int mg_time_coarse_batched(mg_ctx* ctx, int nrhs, int reps, double* ms_per_launch, double* bytes_per_launch,
                           double* flops_per_launch);

/* Coarse stencil (Sec. III) on nrhs coarse vectors at once: y_n = D_c x_n
 * (dagger: D_c^dag).  x, y: nrhs consecutive host coarse vectors, nrhs <= 256.
 * impl 0: tensor cores (operator rounded to FP16 without scale, each source
 * scaled to max |x| = 1 and split into FP16 hi + lo, FP32 accumulation; needs
 * 2 nvec a multiple of 16 and <= 128); impl 1: SIMT with the FP64 operator. */
int mg_apply_coarse_batched(mg_ctx* ctx, const double* x, double* y, int nrhs, int dagger, int impl);

/* ---- single steps of the method (host buffers, FP64 at the boundary; the
 * ---- kernel runs in precision prec) -------------------------------------- */

/* out = D in, eq. (2).  MG_FP16: in rounded to FP16 with a per-site scale,
 * FP16 links, out rounded likewise (the smoother's storage). */
int mg_apply_dslash(mg_ctx* ctx, const double* in, double* out, int prec);

/* r_c = P^dag r: the restriction of the coarse-grid correction (eq. 5 with
 * R = P^dag once the gamma5 factors cancel, chirality kept, Sec. III). */
int mg_restrict(mg_ctx* ctx, const double* r, double* rc, int prec);

/* e = P y_c: prolongation of a coarse vector (eq. 5, Sec. III). */
int mg_prolong(mg_ctx* ctx, const double* yc, double* e, int prec);

/* y = D_c x, or D_c^dag x = sigma3 D_c sigma3 x when dagger != 0 (the coarse
 * operator keeps gamma5-hermiticity as sigma3-hermiticity, Sec. III). */
int mg_apply_coarse(mg_ctx* ctx, const double* x, double* y, int dagger, int prec);

/* nsteps MR smoothing steps (GMRES(1) restarts with under-relaxation omega,
 * the smoother of Sec. III) on (e, r): q = D r, alpha = omega <q,r>/<q,q>,
 * e += alpha r, r -= alpha q.  e and r are read and overwritten.  MG_FP16:
 * r and q stored in FP16 with a per-site scale, FP16 links, e in FP32. */
int mg_mr(mg_ctx* ctx, double* e, double* r, int nsteps, int prec);

/* Coarse solve y = CGNR(D_c, rc) from y = 0 to ||rc - D_c y|| <= tol ||rc||
 * or maxit iterations (tol = 0: exactly maxit): CG on the normal equations,
 * the coarsest-grid solver of Sec. IV.  rc, y: host coarse vectors; *iters
 * and *final_rel (may be NULL) receive the iterations and the final relative
 * coarse residual. */
int mg_coarse_solve(mg_ctx* ctx, const double* rc, double* y, double tol, int maxit, int prec,
                    int* iters, double* final_rel);

/* Allocation-free coarse solve.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they call
 * -- code running under another framework that owns the device allocator, or
 * from a context where cudaMalloc is not allowed or would synchronise the
 * device.  It computes what mg_coarse_solve computes in FP64 (CGNR on the
 * context's D_c from y = 0, same kernels), with rc_dev and y_dev device
 * buffers of Vc * 2 Nv complex doubles (boundary coarse-vector layout) that
 * the caller owns.  It calls no cudaMalloc/cudaFree and no allocating library
 * routine: its work vectors, reduction partial sums and scalars live in one
 * file-scope __device__ array of 6 * 65536 complex doubles plus about 640 KB,
 * which every GPU that loads this library holds until the process exits.
 *   - Sizes: Vc * 2 Nv must be <= 65536, else MG_ERR_INVALID_ARG.
 *   - The first call on a device looks up the array's device address on that
 *     (current) device; make that first call before any stream capture.
 *   - All calls share the one array and it keeps the last call's contents:
 *     the arrival counter is cleared on every call, everything else is
 *     written before it is read.  Calls that overlap on the GPU (other
 *     streams, other host threads, other contexts on the same device) race.
 *   - Work runs on the context's stream; the call synchronises that stream.
 *   - The context's device (current at mg_create) must be current, else
 *     MG_ERR_INVALID_ARG. */
int mg_coarse_solve_noalloc(mg_ctx* ctx, const double* rc_dev, double* y_dev, double tol, int maxit, int* iters,
                            double* final_rel);

/* z = M r, one two-level V(0, smoother_steps) cycle (Sec. II-III: coarse
 * correction with R = P^dag, then post-smoothing; the preconditioner of the
 * flexible GCR).  r, z: host fine spinors. */
int mg_vcycle(mg_ctx* ctx, const double* r, double* z, int prec);

/* Device-resident application of eq. 2 for timing (a measurement hook, no
 * counterpart in the paper): out = D in on internal
 * buffers of the context, `reps` launches, returns the mean kernel time in
 * ms (CUDA events on the context stream) and the bytes one launch must move
 * at minimum (algorithmic: links + input + output, each read/written once). */
int mg_time_dslash(mg_ctx* ctx, int prec, int reps, double* ms_per_launch, double* bytes_per_launch);

/* Latency floor of the on-chip coarse CGNR (measurement hook; the paper has no
 * counterpart).  On the current level-1 operator and the solver's own launch
 * shape, times `rounds` rounds of (a) the two epoch-tagged stencils of one
 * Chronopoulos-Gear iteration without its exchange and (b) its three-value
 * grid exchange alone, each in one cooperative launch (CUDA events on the
 * context's stream, launch overhead included once).  *us_stencils and
 * *us_exchange: microseconds per round.  Needs MG_FP32 or MG_FP16 inner
 * precision and an on-chip shape (MG_ERR_INVALID_ARG otherwise); overwrites
 * the coarse CG work vectors.  MG_ERR_TIMEOUT if a bounded wait gave up. */
int mg_time_coarse_floor(mg_ctx* ctx, int rounds, double* us_stencils, double* us_exchange);

/* As mg_time_dslash (eq. 2), with the L2 cache flushed before every launch: the
 * caller's device buffer `flush` (flush_bytes, larger than the L2) is
 * overwritten on the context stream between launches, and only the dslash
 * launches are timed (one event pair each). */
int mg_time_dslash_cold(mg_ctx* ctx, int prec, int reps, void* flush, size_t flush_bytes, double* ms_per_launch,
                        double* bytes_per_launch);

/* Kernel classes for the launch timer below (steps of Sec. II-IV). */
enum mg_kernel_class {
    MG_K_DSLASH = 0,       /* fine Wilson operator, all variants and precisions */
    MG_K_COARSE_SOLVE = 1, /* persistent CGNR on D_c (whole coarse solve per launch) */
    MG_K_RESTRICT = 2,
    MG_K_PROLONG = 3,
    MG_K_BLOCK_ORTHO = 4,
    MG_K_COARSE_BUILD = 5,
    MG_K_KRYLOV = 6,       /* GCR orthogonalisation, updates, norms, MR updates */
    MG_K_TRUE_RESIDUAL = 7,/* FP64 b - D x at GCR restarts */
    MG_K_NCLASSES = 8
};

/* Launch timer (a measurement hook, no counterpart in the paper): while
 * enabled, every launch of a tracked kernel class is
 * bracketed by CUDA events on the context stream (negligible device cost).
 * mg_profile_read synchronises the stream and returns, per class, the summed
 * device time (ms) and the launch count since the last read (then resets);
 * ms and launches point to MG_K_NCLASSES entries.  *coarse_iters receives
 * the coarse CG iterations run since the last read (profiling on or off). */
int mg_profile_enable(mg_ctx* ctx, int on);
int mg_profile_read(mg_ctx* ctx, double* ms, int* launches, double* coarse_iters);
/* Kernel classes the launch timer tracks while enabled: bit c of mask selects
 * class c (MG_K_*); default all.  Tracking one class keeps the event records
 * off the others' launches.  MG_ERR_INVALID_ARG for a mask with no class. */
int mg_profile_classes(mg_ctx* ctx, unsigned int mask);

/* Number of kernel launches this library has issued in the process so far
 * (all contexts); the difference over a region counts its launches (a
 * measurement hook, no counterpart in the paper). */
long long mg_kernel_launches(void);

/* Which coarse CGNR kernel the last coarse solve of this context ran (a
 * diagnostic; no counterpart in the paper): MG_CK_REGISTER operator read from
 * global memory every iteration, MG_CK_SMEM operator resident in shared
 * memory, MG_CK_STREAM operator streamed through a shared-memory ring,
 * MG_CK_TMEM operator resident in tensor memory, products on the CUDA cores,
 * MG_CK_TMEM_MMA operator resident in tensor memory, products on the tensor
 * cores; MG_CK_NONE before any. */
enum mg_coarse_kernel_id {
    MG_CK_NONE = -1, MG_CK_REGISTER = 0, MG_CK_SMEM = 1, MG_CK_STREAM = 2, MG_CK_TMEM = 3, MG_CK_TMEM_MMA = 4
};
int mg_coarse_kernel(mg_ctx* ctx);

/* Check of the library's bounded device waits (the paper has no counterpart;
 * every spin-wait in these kernels gives up after a poll limit, raises the
 * context's error flag and returns instead of hanging).  Runs one small kernel
 * that drives one wait primitive into a configuration that cannot complete,
 * with a poll limit of spin_limit (1 .. 1e7): kind 0 the epoch exchange of the
 * on-chip coarse CG (one publishing CTA missing), 1 the counter grid barrier of
 * the persistent CG (one arrival missing), 2 an mbarrier transaction that no
 * copy completes, 3 an epoch-tagged vector entry never written.  Returns
 * MG_ERR_TIMEOUT when the wait gave up as designed (the context stays usable),
 * MG_OK if it unexpectedly completed, another status on a CUDA error. */
int mg_check_wait_timeout(mg_ctx* ctx, int kind, long long spin_limit);

/* Name of a status code; last error message of a context (NUL-terminated,
 * owned by the library: valid until the next call on that context).  No
 * counterpart in the paper. */
const char* mg_status_string(int status);
const char* mg_last_error(const mg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* WILSON_MG_H */
