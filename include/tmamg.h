/*
 * tmamg -- simultaneous multi-rhs, multi-shift inversion of the degenerate
 * twisted-mass Wilson-clover Dirac operator with aggregation-based
 * domain-decomposition adaptive multigrid (method of arXiv:2201.03872,
 * "Implementation of Simultaneous Inversion of a Multi-shifted Dirac Matrix
 * for Twisted-Mass Fermions within DDalphaAMG"), on one NVIDIA GB300 (sm_103a).
 *
 * C ABI. Plain pointers and sizes only. Every entry point returns an int
 * status (tmamg_status); a negative value is an error whose text is returned
 * by tmamg_last_error(ctx). Argument checks run before any launch; nothing
 * aborts the process. All device work is ordered on the CUDA stream given to
 * tmamg_create (the calls are asynchronous with respect to the host unless
 * stated otherwise).
 *
 * Operator (paper, Fig. 6 caption: D_TM = D_W + i (delta mu) mu gamma5):
 *   D(mu) x(s) = 1/(2 kappa) x(s) + c_sw C(s) x(s) + i mu gamma5 x(s)
 *               - 1/2 sum_nu [ (1 - gamma_nu) U_nu(s) x(s+nu) + (1 + gamma_nu) U_nu(s-nu)^+ x(s-nu) ]
 * chiral gamma basis: gamma_k = [[0, -i sigma_k], [i sigma_k, 0]], gamma_4 = [[0,1],[1,0]],
 * gamma5 = diag(1,1,-1,-1); C = (i/4) sum_{mu,nu} sigma_{mu nu} F_{mu nu} with the
 * clover-leaf F = (Q - Q^+)/8; periodic in x, y, z, phase bc_t on hops that wrap in t.
 *
 * Layouts.
 *   user vector ("field"): complex numbers [nvec][Lt][Lz][Ly][Lx][spin 4][colour 3],
 *       interleaved (re, im), double or float; x fastest; spin-major inside a site.
 *   gauge field: complex double [Lt][Lz][Ly][Lx][mu 4][3][3], row-major 3x3, mu = x, y, z, t.
 *   bundle (the library's working layout, paper Sec. 3 / Fig. 2: the system index runs
 *       fastest): real [ntile][ncomp][nsite][2 (re, im)][T], with T = 2 systems per tile
 *       in FP32 and T = 1 in FP64 (one 16-byte entry holds re[T], im[T]),
 *       ntile = ceil(nsys / T); system n sits in tile n / T, lane n % T. Fine level:
 *       ncomp = 12 (spin * 3 + colour), nsite = V. Padding lanes of the last tile are
 *       carried along and ignored.
 */
#ifndef TMAMG_H
#define TMAMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tmamg_ctx tmamg_ctx;

typedef enum {
  TMAMG_OK = 0,
  TMAMG_NOT_CONVERGED = 1,  /* soft: x and per-system stats are still written */
  TMAMG_ERR_ARG = -1,       /* invalid argument; nothing was launched */
  TMAMG_ERR_STATE = -2,     /* call out of order (e.g. solve before setup) */
  TMAMG_ERR_OOM = -3,       /* device allocation failed */
  TMAMG_ERR_CUDA = -4,      /* a CUDA call or launch failed */
  TMAMG_ERR_NONFINITE = -5, /* a NaN/Inf was found in an input or iterate */
  TMAMG_ERR_TIMEOUT = -6    /* a bounded device wait gave up */
} tmamg_status;

/* Multigrid setup parameters (paper Sec. 2; defaults by tmamg_default_setup_params). */
typedef struct {
  int levels;          /* 2 (fine + one coarse level) or 3 (a second coarse level on the lattice of level 1) */
  int agg[2][4];       /* aggregate extents (x, y, z, t) for the level-1 and level-2 coarsening */
  int nv[2];           /* test vectors per coarsening; coarse site carries 2*nv unknowns (chirality split) */
  int sap_block[4];    /* SAP block extents on the fine level; block counts per dimension must be even */
  int sap_cycles;      /* red+black sweeps per SAP application */
  int sap_mr_steps;    /* minimal-residual steps per block solve */
  int setup_iters;     /* inverse-iteration steps v <- SAP(v)/|SAP(v)| on the test vectors (on level 1
                          for levels == 3: w <- G(w)/|G(w)|, G = setup_gmres_steps steps of level-1 GMRES) */
  double mu_setup;     /* twisted mass used during setup */
  uint64_t seed;       /* start vectors when none are passed (counter-based splitmix64 + Box-Muller) */
  int setup_gmres_steps; /* levels == 3: Arnoldi steps (<= 64) of the level-1 GMRES that serves as the approximate
                            inverse in the inverse iteration of the level-2 test vectors */
} tmamg_setup_params;

/* Solve parameters (paper Sec. 4: FGMRES at the top, goal residual 1e-10; tuned coarse residual 1e-1). */
typedef struct {
  double tol;          /* per-system true FP64 relative residual goal ||b - D x|| / ||b|| */
  int restart;         /* inner FP32 FGMRES cycle length between FP64 residual recomputations */
  int max_outer;       /* maximum FP64 refinement cycles */
  double coarse_tol;   /* relative residual goal of the coarsest-level solve (r_b) */
  int coarse_restart;  /* coarse GMRES restart length */
  int coarse_maxiter;  /* coarse iterations per cycle, upper bound */
  int coarse_solver;   /* 0: persistent GMRES (one cooperative launch per coarse solve, all systems);
                          1: block GMRES over the rhs of each shift; 2: GMRES with one launch per step */
  double delta_mu;     /* twisted-mass factor of the bottom level's operator, D_c + i delta_mu mu gamma5_c
                          (paper Fig. 6 caption); the finer levels keep mu. 1 = none */
  int precision;       /* 32: the batched mixed-precision solver (FP32 inner FGMRES and AMG cycle, FP16 coarse
                          operands, FP64 refinement); 64: the plain comparator, FGMRES(restart) with the same
                          two-level AMG cycle where every vector, operator and reduction is FP64 (coarse GMRES
                          with one launch per step, no refinement loop, no learned step, coarse_solver and
                          coarse_precision ignored), restarted until the true FP64 residual meets tol */
  int use_nn;          /* learned step in the AMG cycle: 0 off, 1 if trained and enabled by the gate, 2 forced */
  int poll;            /* coarse iterations between host convergence polls */
  int coarse_precision; /* coarse stencil: 16 (default; 0 means 16) FP16 operator and FP16-staged vectors on
                           the tensor cores (tcgen05) with FP32 accumulation, per-system scaling that keeps
                           the FP16 range; 32: FP32 operator on the CUDA cores (reference path) */
  /* levels == 3 (paper Sec. 4: FGMRES on the middle level to r_m, about 7e-2): the level-1 system of every
     AMG cycle is solved by FGMRES(mid_restart) to the relative residual mid_tol (at most mid_maxiter steps),
     preconditioned by the level-2 correction z = P2 D_c2^{-1} P2^+ v (the coarse solver above, to coarse_tol)
     followed by mid_smooth minimal-residual steps on the level-1 residual v - D_c1 z */
  double mid_tol;
  int mid_restart;     /* <= 64 */
  int mid_maxiter;
  int mid_smooth;      /* 0 = no level-1 smoothing */
  int inner_cycles;    /* FP32 FGMRES(restart) cycles per FP64 refinement cycle (>= 1): after each cycle the
                          systems that missed the inner goal restart from their FP32 residual, so the FP64
                          residual (the expensive product on GB300) is formed only once per inner_cycles cycles */
  int sap_cycles;      /* SAP smoother of the solve's AMG cycle: red+black cycles and MR steps per block solve;
                          0 takes the setup's values (tmamg_setup_params sap_cycles, sap_mr_steps), which the
                          setup's own smoothing of the test vectors always uses */
  int sap_mr_steps;
} tmamg_solve_params;

typedef struct {
  int status;          /* TMAMG_OK, TMAMG_NOT_CONVERGED or TMAMG_ERR_NONFINITE for this system */
  int outer_iters;     /* FP64 refinement cycles */
  int inner_iters;     /* top-level FGMRES iterations (= AMG cycles) */
  int coarse_iters;    /* coarse-level iterations summed over all cycles */
  double true_rel_res; /* final ||b - D x|| / ||b|| recomputed in FP64 */
} tmamg_system_stats;

void tmamg_default_setup_params(tmamg_setup_params* p);
void tmamg_default_solve_params(tmamg_solve_params* p);

/* Create a context for an Lx x Ly x Lz x Lt lattice (L[0..3] = x, y, z, t; each even, >= 2).
 * bc_t: -1 antiperiodic or +1 periodic in t. cuda_stream: a cudaStream_t (NULL = default stream).
 * The context owns every device buffer it allocates; tmamg_destroy frees them. */
int tmamg_create(const int L[4], int bc_t, void* cuda_stream, tmamg_ctx** out);
int tmamg_destroy(tmamg_ctx* ctx);
const char* tmamg_last_error(const tmamg_ctx* ctx);
int tmamg_volume(const tmamg_ctx* ctx, int64_t* V);

/* Number of CUDA kernels this library has launched since it was loaded (all contexts). */
uint64_t tmamg_kernel_launches(void);

/* Copy a gauge field (complex double, layout above) into the library's own FP64 and FP32
 * copies. on_device: 1 if U is a device pointer, 0 for host memory. The caller keeps U. */
int tmamg_load_gauge(tmamg_ctx* ctx, const double* U, int on_device);

/* Set kappa and c_sw and build the clover term on the device (FP64, then an FP32 copy).
 * Requires a loaded gauge field. */
int tmamg_set_operator(tmamg_ctx* ctx, double kappa, double c_sw);

/* Bytes of a bundle holding nsys fine-level systems at precision prec (32 or 64). */
size_t tmamg_bundle_bytes(const tmamg_ctx* ctx, int nsys, int prec);

/* Convert between user fields and bundles, device to device. x_field: [nsys][V][4][3]
 * complex (double if prec == 64, float if prec == 32). Padding lanes are zeroed by pack. */
int tmamg_pack(tmamg_ctx* ctx, const void* x_field, void* x_bundle, int nsys, int prec);
int tmamg_unpack(tmamg_ctx* ctx, const void* x_bundle, void* x_field, int nsys, int prec);

/* y = D(mu_n) x_n for every system n, bundles on the device (the fine stencil; paper
 * Sec. 3: the gauge and clover data are loaded once for all systems). mu: host array of
 * nsys twisted masses. prec: 32 or 64. x and y must not overlap. */
int tmamg_dirac(tmamg_ctx* ctx, const void* x_bundle, void* y_bundle, int nsys, const double* mu, int prec);

/* The non-degenerate twisted-mass doublet (paper Sec. 1, the generalisation of the method to a
 * flavour doublet): D_ND(mu, eps) = D_W (x) 1 + i mu gamma5 (x) tau3 - eps 1 (x) tau1, acting on a
 * pair (u, d) of fields as (D(mu) u - eps d, D(-mu) d - eps u), with D(mu) the degenerate
 * operator above. Doublet q occupies systems 2q (u) and 2q + 1 (d) of the bundles: at prec 32
 * one tile of two systems per doublet, at prec 64 the tiles 2q and 2q + 1. mu, eps: host arrays
 * [npair]. x and y (device bundles of 2 npair systems) must not overlap. */
int tmamg_dirac_doublet(tmamg_ctx* ctx, const void* x_bundle, void* y_bundle, int npair, const double* mu,
                        const double* eps, int prec);

/* The even-odd (Schur complement) form of D(mu) (the standard reduction of the DDalphaAMG family the
 * paper builds on, Sec. 2): with the sites split by parity (x + y + z + t) mod 2 the hops connect
 * opposite parities only, and y_n = M_ee(mu_n) x_n = A_ee x_e - H_eo A_oo(mu_n)^{-1} H_oe x_e on the
 * even sites, A the site-local part (diagonal, clover, twist) and H the hops; y is zero on the odd
 * sites and x's odd entries are ignored. The inverse of M_ee is the even block of D^{-1}. Bundles on
 * the device as for tmamg_dirac (nsys systems, prec 32 or 64, mu host [nsys]); uses the context's two
 * scratch bundles; x and y must not overlap. */
int tmamg_dirac_eo(tmamg_ctx* ctx, const void* x_bundle, void* y_bundle, int nsys, const double* mu, int prec);

/* Convenience: y = D(mu_n) x_n on user fields (device pointers), packing through
 * internal scratch bundles. */
int tmamg_apply(tmamg_ctx* ctx, const void* x_field, void* y_field, int nsys, const double* mu, int prec);

/* ------------------------------------------------------------------ multigrid and solve */

/* Build the multigrid hierarchy (paper Sec. 2: test vectors approximating low modes, P and
 * R = P^+ on aggregates, coarse operator D_c = P^+ D P, applied recursively for a further
 * level). start_vectors: device pointer to nv[0] complex float fields [nv][V][4][3], or NULL
 * to draw them from the library's counter-based generator (splitmix64 + Box-Muller, seeded by
 * p->seed). The start vectors are smoothed by p->setup_iters steps of inverse iteration
 * v <- SAP(v)/|SAP(v)| at twisted mass p->mu_setup, split by chirality and orthonormalised
 * per aggregate (classical Gram-Schmidt, twice).
 * levels == 3: the array continues with nv[1] level-1 fields, complex float [nv1][Vc1][2 nv[0]]
 * (level-1 sites lexicographic, x fastest; coarse component chi * nv[0] + j), smoothed by
 * p->setup_iters steps of w <- G(w)/|G(w)| with G = p->setup_gmres_steps steps of level-1
 * GMRES at p->mu_setup, split by the chirality of gamma5_c and orthonormalised per level-2
 * aggregate (extents agg[1], dividing the level-1 lattice); D_c2 = P2^+ D_c1 P2.
 * Synchronises the stream. */
int tmamg_setup(tmamg_ctx* ctx, const tmamg_setup_params* p, const float* start_vectors);

/* As tmamg_setup, but test_vectors (device, complex float [nv][V][4][3], followed for
 * levels == 3 by the level-1 fields described above) are used as the final test vectors
 * without smoothing: lets a caller reproduce P (and P2) from known vectors. */
int tmamg_setup_from_vectors(tmamg_ctx* ctx, const tmamg_setup_params* p, const float* test_vectors);

/* Solve D(mu_k) x_{r,k} = b_r for every rhs r < nrhs and shift k < nshift (paper Sec. 3-4).
 * b: complex double [nrhs][V][4][3]; mu: host array [nshift]; x: complex double
 * [nrhs][nshift][V][4][3]. on_device: 1 if b and x are device pointers, 0 for host memory.
 * p: NULL for defaults. stats: host array [nrhs * nshift] or NULL. Every system is iterated
 * until ||b - D x|| <= p->tol ||b|| in FP64 (or p->max_outer refinement cycles). Returns
 * TMAMG_OK if all systems converged, TMAMG_NOT_CONVERGED otherwise (x and stats written;
 * a system whose data became non-finite has status TMAMG_ERR_NONFINITE and is frozen).
 * Synchronises the stream. */
int tmamg_solve(tmamg_ctx* ctx, const double* b, int nrhs, const double* mu, int nshift, double* x, int on_device,
                const tmamg_solve_params* p, tmamg_system_stats* stats);

/* Solve D_ND(mu_k, eps_k) (x_u, x_d)_{r,k} = (b_u, b_d)_r for the non-degenerate doublet (see
 * tmamg_dirac_doublet) with the same multigrid hierarchy: every level applies the doublet form
 * (the coarse operator of D_ND is D_c(mu) (x) 1 - eps 1 (x) tau1 on P (x) 1, with the coarse
 * twisted mass taking the sign of the flavour), and the Krylov scalars of each doublet are shared
 * by its two flavours. b: complex double [nrhs][2][V][4][3] (flavour u, then d); mu, eps: host
 * arrays [nshift]; x: complex double [nrhs][nshift][2][V][4][3]. stats: host array
 * [nrhs * nshift] (one entry per doublet, norms over both flavours) or NULL. Requires the
 * mixed-precision solver (p->precision 32) with the per-launch coarse GMRES (coarse_solver 0 is
 * taken as 2; 1 and the learned step are rejected). Returns as tmamg_solve; at most 128
 * doublets (rhs x shift) per call. Synchronises the stream. */
int tmamg_solve_doublet(tmamg_ctx* ctx, const double* b, int nrhs, const double* mu, const double* eps, int nshift,
                        double* x, int on_device, const tmamg_solve_params* p, tmamg_system_stats* stats);

/* ------------------------------------------------------------------ learned preconditioner step */
/* A gauge-covariant network of three linear parallel-transport layers (4 -> 8 -> 8 -> 4
 * complex channels of colour 3-vectors; layer out_a(x) = sum_h sum_b W_h[a][b] (T_h in_b)(x)
 * over the identity and the eight link hops T_{+-nu}), applied as an extra step of the AMG
 * cycle: z += N(v - D z) after the smoother. Not part of the paper; trained on (residual,
 * error) pairs from the plain solver. Weights on the host: complex double, the three layers'
 * [9][cout][cin] arrays concatenated (1152 complex numbers). */
typedef struct {
  int pairs;         /* training pairs (a multiple of batch is used) */
  int batch;         /* systems per training batch (<= 16) */
  int epochs;
  double lr;         /* Adam learning rate */
  double pair_tol;   /* relative residual of the solves that produce the errors */
  double mu;         /* twisted mass of the training pairs and of the gate solve */
  uint64_t seed;
  int gate_systems;  /* right-hand sides of the gate solve (<= 16) */
  int window;        /* training batches resident at once (0 = all): the pairs are collected and trained
                        window by window, `epochs` Adam passes over each window, so the pair count is not
                        bounded by device memory */
} tmamg_nn_params;

typedef struct {
  double loss_first, loss_last;  /* mean loss per pair in the first pass over the first window and in the
                                    last pass over the last window (the first and last epoch if one window) */
  int iters_plain, iters_nn;     /* FGMRES iterations of the gate solve without / with the step */
  int enabled;                   /* 1 if the step lowered the iteration count and stays on */
} tmamg_nn_report;

void tmamg_default_nn_params(tmamg_nn_params* p);
/* Start weights: a Jacobi-like map (2 kappa on the spins) plus small seeded noise. */
int tmamg_nn_init(tmamg_ctx* ctx, uint64_t seed);
int tmamg_nn_set_weights(tmamg_ctx* ctx, const double* W);
int tmamg_nn_get_weights(const tmamg_ctx* ctx, double* W);
/* y = N(r) on FP32 fine bundles (4 channels = the 4 spins); bf16: use the BF16 inference weights. */
int tmamg_nn_forward(tmamg_ctx* ctx, const void* r_bundle, void* y_bundle, int nsys, int bf16);
/* loss = sum_n |N(r_n) - e_n|^2 / |e_n|^2 and its gradient (complex double, weight layout). */
int tmamg_nn_loss_grad(tmamg_ctx* ctx, const void* r_bundle, const void* e_bundle, int nsys, double* loss,
                       double* grad);
/* Collect pairs (r = residual after the plain cycle of a random vector, e = D^{-1} r), train
 * with Adam on the GPU, then run the gate: one solve with and one without the step; the step
 * stays enabled (for use_nn = 1) only if it lowered the iteration count. Needs a setup. */
int tmamg_nn_train(tmamg_ctx* ctx, const tmamg_nn_params* p, tmamg_nn_report* report);

/* ------------------------------------------------------------------ components (bundles, device) */

/* Bytes of a coarse bundle of `level` (1 = first coarse level) holding nsys systems (FP32):
 * real [ntile][2 nv][Vc][2][2], coarse component chi * nv + j, coarse sites lexicographic. */
size_t tmamg_coarse_bundle_bytes(const tmamg_ctx* ctx, int level, int nsys);

/* e = SAP(r) on FP32 fine bundles (paper Sec. 2, red-black Schwarz alternating procedure):
 * block extents block[4] (an even number of blocks, or one, per dimension; block volume
 * <= 256), `cycles` red+black sweeps, `mr_steps` minimal-residual steps per block solve,
 * zero start. r is overwritten (partially updated residual). mu: host [nsys], nsys <= 256. */
int tmamg_sap(tmamg_ctx* ctx, void* r_bundle, void* e_bundle, int nsys, const double* mu, const int block[4],
              int cycles, int mr_steps);

/* Fixed limits of tmamg_sap_noalloc: scratch bytes (one FP32 fine bundle) and systems per call. */
#define TMAMG_SAP_NOALLOC_MAX_BYTES ((size_t)64 << 20)
#define TMAMG_SAP_NOALLOC_MAX_SYSTEMS 64

/* tmamg_sap for callers that cannot allocate device memory at call time: code that runs
 * while a stream is being captured into a CUDA graph (cudaMalloc is not allowed there), code
 * that must not touch the allocator after it has fixed its memory budget, or code running
 * under a memory pool it does not own. The paper has no counterpart; this is a property of
 * the library only. Same arguments and arithmetic as tmamg_sap (r is overwritten with the
 * partially updated residual, e receives the correction).
 * Unlike tmamg_sap it does not wait for the stream: the work is queued on the context's
 * stream and the call returns; e and r are written when the stream reaches that work, so a
 * caller reading them from the host or from another stream must synchronise with the
 * context's stream first. The return value reports argument errors and launch errors only;
 * a fault while the kernels run surfaces at a later synchronising call.
 * Its scratch (the correction buffer of the red/black sweeps, and the nsys twisted masses)
 * lives in file-scope device arrays of TMAMG_SAP_NOALLOC_MAX_BYTES bytes and
 * TMAMG_SAP_NOALLOC_MAX_SYSTEMS doubles, which every GPU that loads the library holds until
 * the process exits; the call allocates and frees nothing. A bundle larger than the scratch
 * (ceil(nsys/2) * 12 * V * 16 bytes > TMAMG_SAP_NOALLOC_MAX_BYTES) or more systems than the
 * limit is rejected with TMAMG_ERR_ARG before anything is launched.
 * The first call on a device looks up the arrays' device addresses (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream capture. Every call
 * shares the arrays, which keep the last call's contents: two calls whose work overlaps on
 * the GPU (different streams, or different contexts on one device) race on them.
 * mu: host [nsys], copied into the device array by cudaMemcpyAsync on the context's stream.
 * From pageable memory that copy is staged before the call returns; from page-locked memory
 * the caller keeps mu unchanged until the stream has passed the call. */
int tmamg_sap_noalloc(tmamg_ctx* ctx, void* r_bundle, void* e_bundle, int nsys, const double* mu, const int block[4],
                      int cycles, int mr_steps);

/* xc = P^+ r (restriction) and r = P xc (prolongation, overwrites) between level - 1 (0 = the
 * fine level: fine bundles) and coarse level `level` (1 or, with three levels, 2), FP32 bundles.
 * Require a setup. */
int tmamg_restrict(tmamg_ctx* ctx, int level, const void* fine_bundle, void* coarse_bundle, int nsys);
int tmamg_prolong(tmamg_ctx* ctx, int level, const void* coarse_bundle, void* fine_bundle, int nsys);

/* y = D_c(mu_n) x on coarse level `level` (1 or 2) (9-point stencil of dense 2nv x 2nv blocks plus
 * i mu_n gamma5_c, paper Sec. 2 and Fig. 6 caption with delta mu = 1). mu: host [nsys].
 * precision 16: FP16 stencil blocks and FP16-staged x on the tensor cores, FP32 accumulation;
 * each system's x is scaled by a power of two near 1/max|x_n| before the conversion and y is
 * scaled back, so the elementwise error is about (2^-10 + 18 ncp 2^-22) sum |A_ij| |x_j| over the
 * nine blocks (FP16 rounding of both operands, FP32 sums of 18 ncp terms, ncp = 2nv rounded up
 * to a multiple of 8; 2nv <= 64, at most 1024 systems); precision 32: FP32 blocks on the CUDA
 * cores. Asynchronous on the context stream except for the read of the bounded-wait flag
 * (TMAMG_ERR_TIMEOUT). */
int tmamg_coarse_apply(tmamg_ctx* ctx, int level, const void* x_bundle, void* y_bundle, int nsys, const double* mu,
                       int precision);

/* xc ~ D_c(delta_mu mu_k)^{-1} rc on the bottom coarse level (level 1 of two levels, level 2 of
 * three) by the coarse solver selected in p
 * (p->coarse_solver: 0 persistent GMRES, 1 block GMRES per shift, 2 GMRES with one launch
 * per step; paper Sec. 4), to the relative residual p->coarse_tol per system, restart
 * p->coarse_restart, at most p->coarse_maxiter steps, zero start. Systems n = r * nshift + k
 * (r < nrhs, k < nshift); mu: host [nshift]; rc, xc: coarse bundles of nrhs * nshift
 * systems. iterations (optional): steps taken. With three levels, level 1 is the middle level:
 * FGMRES(p->mid_restart) to p->mid_tol preconditioned by the level-2 correction and
 * p->mid_smooth MR steps (iterations: middle FGMRES steps). Synchronises the stream. */
int tmamg_coarse_solve(tmamg_ctx* ctx, int level, const void* rc_bundle, void* xc_bundle, int nrhs, const double* mu,
                       int nshift, const tmamg_solve_params* p, int* iterations);

/* ------------------------------------------------------------------ diagnostics */

/* Launch-shape autotuning (process-wide, on by default). Kernel families with several launch
 * variants that compute identical results (the fine stencil and its residual forms: CTA shape and
 * register budget) time every variant on the first call for a lattice volume and system count,
 * with CUDA events on that call's stream, and use the fastest from then on (per device). The first
 * call of each shape therefore synchronises its stream once. on = 0 uses the default variant
 * everywhere. Every call clears the recorded choices. Always returns TMAMG_OK. */
int tmamg_autotune(int on);

/* Holds every tuned kernel family to launch variant `variant` (a family with fewer variants uses
 * its default, variant 0), bypassing the tuner; variant < 0 returns to tuning. For checking that
 * the variants agree and for timing one variant. Always returns TMAMG_OK. */
int tmamg_autotune_force(int variant);

/* Writes the choices as NUL-terminated JSON text {"family/devD/key": {"choice": v, "ms": [per
 * variant]}, ...} (key = volume * 4096 + systems). Returns the text length, or TMAMG_ERR_ARG if buf
 * is NULL or len is shorter than the text plus its terminator. */
int tmamg_autotune_report(char* buf, size_t len);

/* Per-kernel timing (process-wide, off by default; no counterpart in the paper). With on != 0
 * the main launch sites of the library (fine stencil and FP64 residual, SAP block solver and
 * face update, restriction, prolongation, coarse stencils, persistent coarse GMRES, the BLAS-1
 * kernels) record a pair of CUDA events on their stream around each launch; every call clears
 * what was recorded. Always returns TMAMG_OK. */
int tmamg_profile_enable(int on);

/* Writes the record as NUL-terminated JSON text {"name": [launches, total_ms], ...} into buf,
 * after waiting for the recorded events. Returns the text length, or TMAMG_ERR_ARG if buf is
 * NULL or len is shorter than the text plus its terminator. */
int tmamg_profile_report(char* buf, size_t len);

/* Failure-path test hook (no counterpart in the paper). Sets, for the whole process, the bound
 * in SM clock cycles of the grid-barrier waits of the persistent coarse GMRES kernel
 * (limit_cycles; 0 restores the default of 2e9 cycles, about one second at 2 GHz). If
 * unreachable_next is nonzero, the next persistent coarse solve (of any context) makes every grid
 * barrier wait for one arrival more than its grid holds, a count that nothing reaches: its first
 * barrier, which follows a plain vector pass, gives up after limit_cycles, the kernel records the
 * failure and returns, and the call reports TMAMG_ERR_TIMEOUT; the request is then cleared.
 * With the FP32 coarse stencil (coarse_precision 32) no bulk copy or tensor-core operation is in
 * flight when the wait gives up. Returns TMAMG_ERR_ARG for limit_cycles < 0. */
int tmamg_debug_bounded_wait(long long limit_cycles, int unreachable_next);

#ifdef __cplusplus
}
#endif

#endif /* TMAMG_H */
