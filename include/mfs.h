/*
 * mfs.h -- C ABI of the GB300 library for the method of fundamental solutions (MFS)
 * with lubrication-adapted image systems for rigid Stokes spheres
 * (Broms, Barnett, Tornberg, arXiv 2407.03343).
 *
 * The library solves the resistance problem of Sec. 1 (eq. stokeseq, eq. bc): P equal
 * rigid spheres with prescribed translational velocities v_k and angular velocities
 * omega_k, optionally in a background flow u_inf, for the disturbance flow
 *     u(x) = sum_k sum_alpha S(x - y^S) f + R(x - y^R) t + D(x - y^D) d      (eq. lin_comb)
 * represented by Stokeslets S on an interior proxy sphere of radius R_p (Sec. 2.1) and
 * Stokeslet/rotlet/potential-dipole triples on the image line of every near contact
 * (Sec. 2.3, Sec. 5.1).  Collocation in the least-squares sense at the surface nodes
 * is solved with one-body right preconditioning (Sec. 2.2, eq. resistance) and GMRES;
 * forces and torques follow from the strengths (Sec. 2.3 remark).
 *
 * Conventions (all calls):
 *  - Every array argument is a HOST pointer owned by the caller unless the function
 *    name ends in _device, in which case it is a device pointer on the context's GPU.
 *    Inputs are copied before the call returns; nothing is retained.
 *  - Coordinates are (x, y, z) triples, row-major: element 3*i + c.
 *  - Calls on a context must follow set_spheres -> build -> set_rigid_velocities (any
 *    time after set_spheres) -> solve -> get_* ; an out-of-order call returns
 *    MFS_ERR_STATE and changes nothing.
 *  - A context is used by one host thread at a time.  Any failure leaves the context
 *    usable, and mfs_last_error() describes it.
 *  - Force sign: F = sum f is the force the sphere exerts on the fluid (Sec. 2.3 remark),
 *    so a sphere translating with U alone has F = +6 pi mu a U.
 *  - All work runs on the context's CUDA stream; calls are synchronous with respect
 *    to the host (they return after the stream has drained) unless stated otherwise.
 */
#ifndef MFS_H
#define MFS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mfs_ctx mfs_ctx;   /* opaque; owns all device memory it allocates */

typedef enum {
  MFS_OK = 0,
  MFS_ERR_ARG = -1,            /* null pointer, size out of range, bad parameter */
  MFS_ERR_GEOMETRY = -2,       /* overlapping or touching spheres */
  MFS_ERR_UNSUPPORTED = -3,    /* e.g. unequal radii */
  MFS_ERR_STATE = -4,          /* call out of order */
  MFS_ERR_NOT_CONVERGED = -5,  /* GMRES / refinement hit its limit; outputs hold the best iterate */
  MFS_ERR_NUMERIC = -6,        /* NaN/Inf or Krylov breakdown */
  MFS_ERR_OOM = -7,            /* device or host allocation failed */
  MFS_ERR_CUDA = -8,           /* a CUDA / cuSOLVER call failed */
  MFS_ERR_TIMEOUT = -9         /* a bounded device wait ran out */
} mfs_status;

/* Precision of the solve and of the single-step entry points:
 *  MFS_FP64   native FP64 everywhere.
 *  MFS_MIXED  GMRES passes with the operator evaluated in double-float arithmetic (pairs of
 *             FP32 values, ~2^-46 relative) on the FP32 pipes, which this GPU executes 74x
 *             faster than FP64: pair sums of steps 2+3 and the pseudo-inverse GEMVs of step 1,
 *             where the GMRES passes read Sigma^+ U^T from its FP32 copy (half the bytes; the
 *             operator stays accurate to ~1e-7, enough for the passes) and V in double-float;
 *             after each pass the residual is re-evaluated with the all-double-float or the
 *             native FP64 operator (mfs_solve_opts.residual) and the correction equation
 *             solved again (iterative refinement).  The single-step entry points with
 *             MFS_MIXED apply the all-double-float operator.
 *  MFS_FP32   FP32 inner GMRES on an all-FP32 operator with FP64 iterative refinement;
 *             converges only when B_k^+ amplifies by well under 1/eps_FP32, i.e. not with
 *             images and the paper's truncation 5e-12 (returns MFS_ERR_NOT_CONVERGED). */
enum { MFS_FP64 = 0, MFS_MIXED = 1, MFS_FP32 = 2 };
/* Single-step entry points only: the operator of the MFS_MIXED GMRES passes themselves (Sigma^+ U^T
 * from its FP32 copy, and the far field when mfs_params.far_dist > 0). */
enum { MFS_MIXED_PASS = 3 };

/* Discretisation parameters (Sec. 2.1, Sec. 2.3, Sec. 5.1, App. A.1).
 * Defaults (mfs_default_params): the paper's coarse choice N = 686, R_p = 0.63,
 * M0 = 823 (~1.2 N), Delta = 0.05, alpha = 6, beta1 = pi/5, beta2 = pi/60,
 * eps_trunc = 5e-12, n_im rule ceil(-8.72 log10(delta) - 6.15) for delta < 0.15,
 * capped at 20, left row scaling on, viscosity 1. */
typedef struct {
  int n_proxy;          /* N: proxy Stokeslets per sphere on radius r_proxy * a */
  double r_proxy;       /* R_p, in radius units, 0 < R_p < 1/(1 + delta_offset) */
  int m_basic;          /* M0: basic collocation nodes per sphere (Fibonacci grid) */
  double delta_offset;  /* Delta in eq. tj */
  int alpha1, alpha2;   /* cap upsampling, eq. colloc_nbr: M_cap = alpha * 3 * n_im */
  double beta1, beta2;  /* cap half-angles (radians), eq. thetacap */
  double eps_trunc;     /* singular values below eps_trunc * sigma_max are dropped */
  double nim_a, nim_b, nim_cut; /* eq. image_est: n_im = ceil(-nim_a log10(delta) - nim_b) if delta < nim_cut */
  int nim_max;          /* cap on n_im (20) */
  int nim_fixed;        /* >= 0: every contact with delta < nim_cut gets exactly this n_im */
  int left_precond;     /* 1: rows scaled by sqrt(area weight) (Sec. 5.1 remark left-precond) */
  double visc;          /* viscosity mu */
  int build_factors;    /* 1 (default): compute the one-body pseudo-inverses; 0: discretise only, after
                           which mfs_apply_pairs and mfs_eval_velocity work but solves and the
                           pseudo-inverse steps return MFS_ERR_STATE */
  int nim_min;          /* at least this n_im for every contact with delta < nim_cut (default 0: the rule as
                           printed, eq. image_est).  Not in the paper: with nim_cut 0.3 and nim_min 2 the
                           gaps 0.15 <= delta < 0.3, where the printed rule places no images and the coarse
                           proxy sphere alone misses the 1e-3 target, get two images each */
  /* Far field of the GMRES passes (not in the paper, which evaluates step 2 with an FMM): with
   * far_dist > 0 a sphere k' whose centre is at least far_dist * a from the target sphere's acts in
   * the MIXED passes through far_n_eq equivalent Stokeslets on radius far_r_eq * a about c_k',
   * whose strengths are q_k' = Q mu_k' with Q = Pinv(S_ce) G_chk B_k'^+ formed once in FP64
   * (S_ce: Stokeslets from the equivalent points to 2 far_n_eq check points on radius far_r_chk * a,
   * pseudo-inverse truncated at far_eps of its largest singular value; G_chk: the sphere's own
   * sources at the check points), so the amplification of B^+ never enters the FP32 sums.
   * Nearer spheres are summed directly in double-float.  The refinement residual always uses
   * every pair directly, so the far field changes how fast the passes run, not the accuracy of
   * the solution.  Needs far_dist >= far_r_chk + 1.  Defaults: far_dist 0 (off), 300, 1.0, 2.0,
   * 1e-6.  Single solves only; batched solves evaluate every pair directly. */
  double far_dist;
  int far_n_eq;
  double far_r_eq;
  double far_r_chk;
  double far_eps;
  /* Step 1 of the MIXED passes for the spheres without contacts, which share the basic factor
   * (Sec. 2.2): 1 (default) as one matrix product on the tensor cores (tcgen05, bf16 slices with
   * FP32 accumulation, the accuracy of the FP32 Sigma^+ U^T those passes use) once at least 8
   * spheres share it, 2 whenever at least one does, 0 never (batched GEMV for every sphere).
   * Applies to Sigma^+ U^T and, with the far field, to Q; single solves and single steps. */
  int tensor_step1;
} mfs_params;

/* GMRES / refinement options (precision as above).  Every mode re-evaluates the residual
 * ||W b - G_hat mu|| / ||W b|| with its FP64-accurate operator after each GMRES pass and
 * solves the correction equation again (iterative refinement) until it is <= tol.
 * Defaults: MIXED, tol 1e-6 (Sec. 3, Sec. 5), max_iter 2000, restart 300,
 * max_refine 20, inner_tol 1e-4 (MFS_FP32 inner solves only). */
typedef struct {
  int precision;
  double tol;
  int max_iter;     /* total inner GMRES iterations over all refinements */
  int restart;      /* GMRES restart length m */
  int max_refine;   /* outer refinement steps (MIXED) */
  double inner_tol; /* relative residual reduction asked of each inner solve (MIXED) */
  int residual;     /* operator of the refinement residual, MFS_RESIDUAL_* below */
} mfs_solve_opts;

/* Operator that evaluates the refinement residual of MFS_MIXED (MFS_FP64 always uses native FP64,
 * MFS_FP32 always the FP64 operator as well):
 *   MFS_RESIDUAL_AUTO   (default) the double-float operator when tol >= MFS_DW_RESIDUAL_MIN_TOL,
 *                       the native FP64 operator for tighter tolerances;
 *   MFS_RESIDUAL_FP64   always the native FP64 operator (FP64 pipes, ~70x slower pair sums);
 *   MFS_RESIDUAL_SOLVE  always the operator of the solve (double-float for MFS_MIXED).
 * The double-float operator's sums are accurate to ~1e-13 of their absolute sums; the massive
 * cancellation of the preconditioned operator (lambda_hat ~ 1e9 |mu|) turns that into a residual
 * floor far below MFS_DW_RESIDUAL_MIN_TOL, so the reported residual stays a faithful measure there. */
enum { MFS_RESIDUAL_AUTO = 0, MFS_RESIDUAL_FP64 = 1, MFS_RESIDUAL_SOLVE = 2 };
#define MFS_DW_RESIDUAL_MIN_TOL 5e-7

typedef struct {
  int iters;           /* GMRES iterations (all refinements) */
  int refinements;     /* outer FP64 residual evaluations after the first */
  double rel_residual; /* final ||W b - G_hat mu|| / ||W b||, evaluated in FP64 */
  double seconds;      /* wall time of the call */
  int converged;       /* 1 if rel_residual <= tol */
} mfs_solve_info;

typedef struct {
  int P;              /* spheres */
  int n_contacts;     /* near contacts that received images */
  int n_colloc;       /* total collocation nodes, sum_k M^(k); operator size is 3*n_colloc */
  int n_proxy_total;  /* P * N */
  int n_image_nodes;  /* total image nodes; each carries S, R and D (3 vector sources) */
  int n_unknowns;     /* 3 * sum_k N^(k) = 3 * (n_proxy_total + 3 * n_image_nodes) */
  int n_factors;      /* distinct one-body factors (shared basic block + one per contact sphere) */
  long long pairs_fp; /* (target node, vector source) pairs of one operator apply, self blocks excluded;
                         an image S+R+D triple counts as 3 */
  long long pairs_near_fp;  /* with the far field: of those, the pairs with near spheres (double-float) */
  long long pairs_far_eq;   /* and the (target node, equivalent Stokeslet) pairs replacing the rest (FP32) */
  int n_factors_shared;     /* factors of spheres without images: these live in a process-wide store
                               per device and are shared with every context whose spheres have the same
                               self block (same radius, viscosity, proxy and collocation grids,
                               truncation and far-field settings), so equal spheres need one SVD across
                               contexts (Sec. 4); each holder counts them in its memory use */
  int n_factors_reused;     /* of those, the factors this build took from the store instead of computing */
} mfs_sizes_t;

void mfs_default_params(mfs_params* p);
void mfs_default_solve_opts(mfs_solve_opts* o);

/* Create a context on CUDA device `device`; `cuda_stream` is a cudaStream_t to run on,
 * or NULL for a stream the context creates and owns. */
mfs_status mfs_create(mfs_ctx** out, int device, void* cuda_stream);
void mfs_destroy(mfs_ctx* ctx);
/* Message of the last failure on this context ("" if none).  Owned by the context. */
const char* mfs_last_error(const mfs_ctx* ctx);

/* P spheres: centres (P*3), radii (P).  All radii must be equal (MFS_ERR_UNSUPPORTED
 * otherwise, Sec. 2.1 fixes identical spheres); spheres must not touch or overlap
 * (MFS_ERR_GEOMETRY).  Invalidates any previous build. */
mfs_status mfs_set_spheres(mfs_ctx* ctx, int P, const double* centres, const double* radii);

/* Rigid-body boundary data of eq. bc: v (P*3), omega (P*3).  Non-finite values give MFS_ERR_ARG
 * (the host variant checks them; device data that is not finite makes the next solve return
 * MFS_ERR_NUMERIC). */
mfs_status mfs_set_rigid_velocities(mfs_ctx* ctx, const double* v, const double* omega);
mfs_status mfs_set_rigid_velocities_device(mfs_ctx* ctx, const double* d_v, const double* d_omega);

/* Mobility problem (the inverse of the resistance problem that the Sec. 2.3 remark on forces
 * and torques makes available): prescribe F (P*3) and T (P*3) on every sphere instead of the
 * rigid velocities; the next mfs_solve then finds mu together with the velocities V_k, Omega_k
 * from the bordered system
 *   G_hat mu - W (V_k + Omega_k x (x - c_k)) = -W u_inf
 *   s_F F_k(B^+ mu) = s_F F_k,   s_T T_k(B^+ mu) = s_T T_k,
 * with s_F = 1/(6 pi visc a) and s_T = 1/(8 pi visc a^3) (the single-sphere drag and torque
 * coefficients, which bring the border rows to the scale of the velocities).  Host arrays,
 * copied before return; non-finite values give MFS_ERR_ARG.  Requires mfs_build.  The mobility
 * problem is solved with MFS_FP64 or MFS_MIXED, singly or in mfs_batch_solve together with
 * resistance problems (MFS_FP32 gives MFS_ERR_UNSUPPORTED; mfs_batch_solve_rhs*, which brings
 * rigid velocities, solves every problem as a resistance problem).  A later
 * mfs_set_rigid_velocities* returns the context to the resistance problem. */
mfs_status mfs_set_forces_torques(mfs_ctx* ctx, const double* F, const double* T);
/* Rigid velocities V (P*3) and Omega (P*3) of the last mobility solve, host arrays;
 * MFS_ERR_STATE before one. */
mfs_status mfs_get_rigid_velocities(mfs_ctx* ctx, double* v, double* omega);

/* Background flow u_inf(x) = U + E x + Omega x x subtracted in eq. bc (Sec. 4, Ex. 2).
 * Each pointer may be NULL (term absent): U (3), E (3*3 row-major), Omega (3).  Non-finite
 * values give MFS_ERR_ARG and leave the previous background flow in place. */
mfs_status mfs_set_background_flow(mfs_ctx* ctx, const double* U, const double* E, const double* Omega);

/* Discretise (contacts, image lines, caps, weights) and compute every distinct
 * one-body truncated pseudo-inverse B_k^+ = V Sigma^+ U^T in FP64 on the GPU
 * (Sec. 2.2, Sec. 2.3, Sec. 5.1).  NULL params = defaults. */
mfs_status mfs_build(mfs_ctx* ctx, const mfs_params* params);
mfs_status mfs_sizes(const mfs_ctx* ctx, mfs_sizes_t* out);

/* The discretisation step of mfs_build alone (Sec. 2.1 basic grids, Sec. 2.3 image lines,
 * Sec. 5.1 n_im rule, caps and weights), on the host, without a context or a GPU: P spheres of
 * radius `radius` at `centres` (P*3), `params` NULL = defaults.  Call once with null arrays to
 * get *n_colloc and *n_sources (vector sources; an image node counts 3), then with arrays of
 * those sizes: x (n_colloc*3), w (n_colloc) and owner (n_colloc) in the layout of
 * mfs_get_collocation, pos (n_sources*3) and type (n_sources) in that of mfs_get_strengths.
 * Any pointer may be NULL.  Returns MFS_ERR_ARG for bad sizes or parameters and
 * MFS_ERR_GEOMETRY for touching or overlapping spheres; nothing is allocated on a device. */
mfs_status mfs_discretise_host(int P, const double* centres, double radius, const mfs_params* params,
                               int* n_colloc, int* n_sources, double* x, double* w, int* owner,
                               double* pos, int* type);

/* Solve eq. resistance for the current boundary data, then form lambda = B^+ mu (FP64, or the
 * double-float factors at ~2^-46 relative accuracy for MFS_MIXED).
 * NULL opts = defaults; info may be NULL.  MFS_ERR_NOT_CONVERGED still leaves the
 * best iterate's outputs available. */
mfs_status mfs_solve(mfs_ctx* ctx, const mfs_solve_opts* opts, mfs_solve_info* info);

/* Forces and torques on each sphere (Sec. 2.3 remark): F (P*3), T (P*3). */
mfs_status mfs_get_forces_torques(mfs_ctx* ctx, double* F, double* T);
mfs_status mfs_get_forces_torques_device(mfs_ctx* ctx, double* d_F, double* d_T);

/* Disturbance velocity u(x) = G(x) lambda at n arbitrary points x (n*3) -> u (n*3),
 * FP64; points inside a sphere get the (meaningless) continuation. */
mfs_status mfs_eval_velocity(mfs_ctx* ctx, int n, const double* x, double* u);

/* Strengths lambda (n_unknowns) in the library's order: per sphere k, first the N proxy
 * Stokeslets (3 each), then per image node its Stokeslet f, rotlet t and dipole d
 * (9 values).  pos (n_vector_sources*3) and type (0 = S, 1 = R, 2 = D) may be NULL. */
mfs_status mfs_get_strengths(mfs_ctx* ctx, double* lambda, double* pos, int* type);

/* Collocation nodes (n_colloc*3), area weights (n_colloc) and owner sphere (n_colloc);
 * per sphere: M0 basic nodes, then for each partner in ascending index order its two caps.
 * Any pointer may be NULL. */
mfs_status mfs_get_collocation(mfs_ctx* ctx, double* x, double* w, int* owner);

/* ---- single steps of the hot path, for checking each against a reference ----
 * Vectors in row space have length 3*n_colloc (node-major, xyz), vectors in source
 * space have length n_unknowns in the strength order above.  All host pointers. */

/* W b: scaled boundary data at the collocation nodes (eq. lq2). */
mfs_status mfs_get_rhs(mfs_ctx* ctx, double* wb);
/* out = G_hat mu (eq. resistance) by the three steps of Sec. 2.2 with steps 2 and 3
 * fused (self blocks skipped), with the operator of the given precision mode. */
mfs_status mfs_apply_operator(mfs_ctx* ctx, int precision, const double* mu, double* out);
/* Step 1 alone: lambda_hat = B_k^+ mu_k for every sphere (eq. transform). */
mfs_status mfs_apply_precond(mfs_ctx* ctx, int precision, const double* mu, double* lambda_hat);
/* Steps 2+3 alone: out = mu + W_k sum_{k' != k} G^(kk') lambda_hat_k' (eq. uAll). */
mfs_status mfs_apply_pairs(mfs_ctx* ctx, int precision, const double* lambda_hat,
                           const double* mu, double* out);

/* ---- step 1 without any device allocation ----
 * The paper has no counterpart to this call; it serves callers that cannot allocate device
 * memory while they run: an application that owns all device memory through its own pool and
 * forbids cudaMalloc/cudaFree (which also synchronise the device) inside its time-stepping
 * loop, or code on a latency-critical path.  It computes the same lambda_hat = B_k^+ mu_k for
 * every sphere as mfs_apply_precond with MFS_FP64, but from DEVICE buffers the caller owns:
 * d_mu (3*n_colloc doubles) in, d_lambda_hat (n_unknowns doubles) out.  The intermediate
 * Sigma^+ U^T mu lives in a fixed array of 2^21 doubles (16 MiB) that the library reserves on
 * every GPU that loads it, until the process exits; a context whose summed retained ranks
 * exceed that size gets MFS_ERR_ARG.  The call allocates nothing (the context's factors were
 * allocated by mfs_build).  Its first call on a device looks up the array's device address;
 * make that first call before any stream capture.  All calls share the one array: calls that
 * overlap on the GPU (other threads, contexts or streams) race and must be serialised by the
 * caller.  Nothing in the array needs clearing; each call overwrites what it reads.  The work
 * runs on the context's stream, which is not ordered after the caller's other streams: d_mu
 * must be complete when the call is made (synchronise the stream that wrote it first, or
 * create the context on that stream with mfs_create).  The array's address is looked up again
 * whenever the calling thread's CUDA context differs from the one of the previous lookup on
 * that device (e.g. after cudaDeviceReset).  Returns after the context's stream has drained. */
mfs_status mfs_apply_precond_noalloc(mfs_ctx* ctx, const double* d_mu, double* d_lambda_hat);

/* ---- many independent problems ----
 * Solves every context (each already built and given boundary data: rigid velocities, or
 * prescribed forces and torques for a mobility problem) with the same options,
 * all at once: one GMRES runs in lockstep over the concatenation of the problems, each with
 * its own Krylov coefficients, Hessenberg matrix and convergence test, and every kernel
 * launch (pseudo-inverse GEMVs, pair sums, Gram-Schmidt) covers all problems still iterating.
 * Restarts are iterative-refinement passes on the true residual.  The work runs on the first
 * context's stream, ordered after work already queued on every context's stream; each
 * context's stream then waits for the batch, and its outputs (forces/torques, strengths,
 * velocity evaluation) are available as after mfs_solve.  MFS_FP32 falls back to solving
 * the problems concurrently on their own streams.  All contexts must be on one device and
 * distinct.  infos (n_problems entries) may be NULL.  Returns MFS_OK if all converged, else
 * the first failing status in problem order; each context keeps its own mfs_last_error. */
mfs_status mfs_batch_solve(int n_problems, mfs_ctx* const* ctxs, const mfs_solve_opts* opts,
                           mfs_solve_info* infos);

/* Several right-hand sides per geometry (a resistance matrix needs 6P of them, a sweep of
 * motions several): problem i is (ctxs[i], v[i], omega[i]) with v[i], omega[i] of P_i*3 values;
 * contexts MAY repeat.  All problems run in one lockstep batch as in mfs_batch_solve, and the
 * pseudo-inverse factors of a repeated context are read once per apply for all its right-hand
 * sides.  Forces and torques of problem i go to F[i], T[i] (P_i*3 each, entries may be NULL);
 * each context afterwards holds the solution of its last problem in the list (for
 * mfs_eval_velocity / mfs_get_strengths).  Background flows are the contexts' own.
 * MFS_FP64 and MFS_MIXED only.  The _device variant takes device pointers for v, omega, F, T. */
mfs_status mfs_batch_solve_rhs(int n_problems, mfs_ctx* const* ctxs, const double* const* v,
                               const double* const* omega, const mfs_solve_opts* opts,
                               mfs_solve_info* infos, double* const* F, double* const* T);
mfs_status mfs_batch_solve_rhs_device(int n_problems, mfs_ctx* const* ctxs, const double* const* d_v,
                                      const double* const* d_omega, const mfs_solve_opts* opts,
                                      mfs_solve_info* infos, double* const* d_F, double* const* d_T);

/* ---- measurement ----
 * With profiling on, the context brackets each launch of the pair kernel (steps 2+3) and of the
 * pseudo-inverse GEMVs (step 1) with CUDA events on its stream and accumulates their device
 * time.  kernel_launches counts every kernel the context launched (profiling on or off). */
typedef struct {
  long long kernel_launches;
  long long pair_launches;       /* operator applies (pair kernel of any precision) */
  double pair_ms;                /* summed device time of those launches */
  long long pair_interactions;   /* sum of pairs_fp over those launches */
  long long pair_proxy;          /* of which (node, proxy Stokeslet) pairs */
  long long pair_image_nodes;    /* and (node, image node) pairs, each an S+R+D triple */
  int pair_kind;                 /* precision of the last pair launch: MFS_FP64, MFS_MIXED or MFS_FP32 */
  long long gemv_launches;
  double gemv_ms;
  double gemv_bytes;             /* factor bytes read by those launches */
  /* the pair statistics split by precision (index MFS_FP64, MFS_MIXED, MFS_FP32) */
  long long by_kind_launches[3];
  double by_kind_ms[3];
  long long by_kind_proxy[3];
  long long by_kind_image_nodes[3];
  /* Gram-Schmidt kernels of the batched GMRES (dot products and updates against the Krylov
   * basis, eq. resistance solved by GMRES): launches, summed device time, and the bytes they
   * must move at the least: a dot product of j basis vectors with w over n active entries reads
   * (j + 1) n doubles, an update w -= sum_i c_i V_i reads (j + 1) n and writes n doubles */
  long long krylov_launches;
  double krylov_ms;
  double krylov_bytes;
  /* far field of the passes: launches of the FP32 equivalent-source kernel, their device time and
   * the (target node, equivalent Stokeslet) pairs they evaluated; the near part of those applies
   * is counted with the pair kernel above (pair_proxy / pair_image_nodes of the near spheres) */
  long long far_launches;
  double far_ms;
  long long far_pairs;
  /* tensor-core step 1 (spheres sharing the basic factor): matrix products launched and the
   * sphere columns they covered */
  long long tc_launches;
  long long tc_columns;
  /* FP32-pipe flops issued by the double-float pair evaluations: 248 per (node, proxy) pair and
   * 544 per (node, image node) triple for one right-hand side; in a batch, the right-hand sides on
   * one geometry (R of them) share each pair's geometry (distance and its powers: 99 and 106
   * flops), so such a pair issues 99 + 149 R (triple: 106 + 438 R).  pair_shared_rhs counts the
   * pair_interactions evaluated that way. */
  double pair_issued_flops;
  long long pair_shared_rhs;
} mfs_timing_t;
mfs_status mfs_set_profiling(mfs_ctx* ctx, int on);
/* Copies the counters; reset != 0 zeroes them afterwards. */
mfs_status mfs_get_timing(mfs_ctx* ctx, mfs_timing_t* out, int reset);

/* Measured CUDA-core arithmetic peak of device `device`, the roofline denominator of the pair
 * kernels (which are bound by FP32-pipe issue, not by a tensor-core contraction): a kernel of
 * independent fused multiply-add chains, 8 per thread, on every SM, timed with CUDA events after
 * a warm-up launch.  which = 0: FP32 FFMA; which = 1: FP64 DFMA.  *tflops receives
 * 2 x FMAs / second / 1e12 (an FMA counts two flops) and *ms the timed launch's duration; the
 * launch runs ~0.1-0.5 s.  Allocates and frees one small device buffer. */
mfs_status mfs_probe_alu_peak(int device, int which, double* tflops, double* ms);

/* Tile shapes of the pair kernels (steps 2+3) and the autotuner that picks them.  A target tile
 * holds 512 collocation nodes (4 per thread of a 128-thread CTA) or 128 (1 per thread); a tile's
 * sources may be split over several CTAs whose partial sums a second kernel adds in a fixed
 * order.  By default the library chooses by rule (512-node tiles once they fill the GPU twice,
 * source parts that fill whole waves of resident CTAs).  mfs_tune_pairs times every candidate
 * (tile of 128 or 512 nodes x no split or the wave-filling split; for the far kernel with 512-node
 * tiles also scalar or packed two-lane FP32 instructions) of each pair-kernel family the
 * context uses, on its own discretisation, with CUDA events over two launches each, keeps the
 * fastest for the context's later launches and reports them; 0 in a field means "not used by
 * this context" (e.g. the near / far kernels without the far field). */
typedef struct {
  int all_nodes_per_thread, all_parts;    /* every pair in double-float (MIXED residual, passes without far field) */
  int near_nodes_per_thread, near_parts;  /* near spheres, double-float (passes with the far field) */
  int far_nodes_per_thread, far_parts;    /* far spheres' equivalent Stokeslets, FP32 */
  int far_packed;                         /* 1: the far kernel issues packed FP32 pairs (f32x2) */
  double all_ms, near_ms, far_ms;         /* device time of the chosen shapes, per launch */
} mfs_pair_shapes;
mfs_status mfs_tune_pairs(mfs_ctx* ctx, mfs_pair_shapes* out);

/* Cap on the device memory the context may hold for its discretisation, factors and solver
 * workspace (bytes; 0 = no cap, the default).  An allocation that would exceed it fails like a
 * cudaMalloc failure: the call returns MFS_ERR_OOM and the context stays usable, so a caller
 * that shares the GPU can keep this library inside its share.  The cap does not cover the
 * transient scratch of the one-body SVDs inside mfs_build nor the workspace of the batched
 * solves (which the first context of a batch holds). */
mfs_status mfs_set_memory_limit(mfs_ctx* ctx, unsigned long long bytes);
/* Device bytes the context currently holds under that accounting. */
mfs_status mfs_memory_in_use(const mfs_ctx* ctx, unsigned long long* bytes);

#ifdef __cplusplus
}
#endif
#endif /* MFS_H */
