/*
 * rve.h -- C ABI of the GB300 linear-finite-element compatibility-projection
 * homogenization solver (Leute et al., "Elimination of ringing artifacts by
 * finite-element projection in FFT-based homogenization").
 *
 * Problem (Sec. 2.1, Eqs. stat-mech-equi2 and stat-mech-equi-FFT-homogenization;
 * small-strain form of Appendix B): a periodic cell of n_x * n_y (* n_z)
 * voxels, each split into linear finite elements (Sec. 2.6: two triangles per
 * pixel in 2D; six Kuhn tetrahedra per voxel in 3D), isotropic small-strain
 * elasticity with a per-voxel Young's modulus and one Poisson ratio (plane
 * strain in 2D).  For a macroscopic strain E the solver finds the compatible,
 * mean-free strain fluctuation eps~ with  G * C : (E + eps~) = 0, where
 * G(k) = B(k) (B(k)^H B(k))^-1 B(k)^H is the projection onto compatible
 * fields built from the Fourier symbols of the element gradient stencils
 * (Eqs. genfourderiv, discrete_projection_op, small-strain-eq2), with
 * G(0) = 0 so that every element keeps the macroscopic strain as its mean
 * (the k = 0 rule of Sec. 2.3).  The solver is a projected conjugate
 * gradient (the gradient-based optimiser of Sec. 2.1).
 *
 * Conventions
 *  - Grid sizes n[0] = n_x, n[1] = n_y (, n[2] = n_z).  Supported: powers of
 *    two, 16..1024 per axis in 2D and 16..256 per axis in 3D.  Other sizes
 *    return RVE_ERR_UNSUPPORTED_SIZE (there is no CPU fallback).
 *  - Per-voxel arrays: x fastest, index v = x + n_x*(y + n_y*z).
 *  - Strain/stress vectors use Mandel notation: 2D (xx, yy, sqrt2*xy),
 *    3D (xx, yy, zz, sqrt2*yz, sqrt2*xz, sqrt2*xy); n_s = 3 or 6.
 *  - A strain FIELD holds m = n_q*n_s scalars per voxel, component-major:
 *    array [m][N] with component c = Theta*n_s + s (element Theta, Mandel s).
 *    Element order: 2D Theta=0 on nodes {00,10,01}, Theta=1 on {11,01,10};
 *    3D Theta = lexicographic index of the permutation (a,b,c) of (x,y,z),
 *    tetrahedron {0, e_a, e_a+e_b, e_a+e_b+e_c}.
 *  - Nodal fields (displacements) hold D scalars per node, [D][N]; node v is
 *    the lower corner of voxel v.
 *  - DFT convention of Appendix A (forward exp(-i k.r), inverse with 1/N).
 *
 * Memory and streams
 *  - A handle owns all of its device memory; caller buffers are borrowed for
 *    the duration of a call only.  Pointers flagged RVE_PTR_DEVICE are device
 *    pointers on the handle's device, otherwise host pointers.
 *  - Work runs on a stream the handle creates; at every call it is ordered
 *    after the work already queued on the stream given to rve_create (NULL =
 *    the legacy default stream), and calls return when their results are
 *    ready (host or device).  A handle must not be used by two host threads
 *    at once.  The CG iterations run as CUDA graphs of 8 iterations.
 *  - Devices: a handle (and a batch) lives on the device that was current at
 *    rve_create (rve_batch_create).  Every call makes that device current for
 *    its duration and restores the caller's current device before it returns,
 *    so handles on several devices can be used from one host thread.  Kernel
 *    attributes are set once per device.  After cudaDeviceReset on a device,
 *    destroy its handles; they are not usable again.
 *
 * Errors: every function returns RVE_OK (0) or a negative code; the text of a
 * code is rve_error_string(code).  After RVE_ERR_CUDA the handle should be
 * destroyed.  RVE_ERR_NOT_CONVERGED leaves readable (unconverged) results.
 */
#ifndef RVE_H
#define RVE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rve_s* rve_t;

enum {
  RVE_OK = 0,
  RVE_ERR_ARG = -1,              /* invalid argument or call order */
  RVE_ERR_UNSUPPORTED_SIZE = -2, /* grid size outside the GPU FFT's range */
  RVE_ERR_CUDA = -3,             /* a CUDA runtime call failed */
  RVE_ERR_OOM = -4,              /* device allocation failed */
  RVE_ERR_NOT_CONVERGED = -5,    /* max_iter reached before the tolerance */
  RVE_ERR_NONFINITE = -6,        /* NaN/Inf or CG breakdown (non-positive curvature) */
  RVE_ERR_TIMEOUT = -7,          /* a device-side wait exceeded its limit */
  RVE_ERR_SCRATCH_LIMIT = -8     /* grid larger than the static scratch of rve_apply_operator_2d_static */
};

enum { RVE_FP64 = 0, RVE_MIXED = 1 };          /* precision of rve_create */
enum { RVE_F32 = 0, RVE_F64 = 1 };              /* dtype codes */
enum { RVE_PTR_HOST = 0, RVE_PTR_DEVICE = 1 };  /* pointer flags */

typedef struct {
  int32_t iterations;     /* projected-CG iterations (summed over refinement steps) */
  int32_t refine_steps;   /* outer FP64 refinement steps (1 for RVE_FP64) */
  int32_t status;         /* RVE_OK or RVE_ERR_NOT_CONVERGED / RVE_ERR_NONFINITE */
  int32_t reserved;
  double rel_residual;    /* final ||f|| / ||f_0|| of the FP64 nodal residual f = B^T C (E + eps~) */
  double cg_rel_residual; /* final relative residual of the last projected-CG solve */
} rve_info;

/* Text of a status code (static storage). */
const char* rve_error_string(int code);

/* Create a solver for a dim-dimensional periodic grid.
 *  n[dim]      voxels per axis (x first);
 *  length[dim] cell edge lengths (NULL = unit cell); voxel size = length/n (Appendix A);
 *  precision   RVE_FP64: every step in FP64.  RVE_MIXED: FFTs, projection and
 *              material in FP32 inside an FP64 iterative refinement on the nodal
 *              displacement (CG scalars and reductions in FP64);
 *  cuda_stream a cudaStream_t (NULL = default stream).
 * The handle runs its work on a non-blocking stream of its own, which every
 * call first orders after cuda_stream (device data the caller wrote there is
 * seen); every call that returns results (solve, means, fields, operator
 * application) returns after its device work has completed.  Calls on one
 * handle must not run concurrently from several host threads.
 * Allocates device memory for one load case; more is allocated by rve_solve. */
int rve_create(rve_t* out, int dim, const int64_t* n, const double* length,
               int precision, void* cuda_stream);

/* Destroy a handle and free its device memory.  NULL is accepted. */
int rve_destroy(rve_t h);

/* Set the material: per-voxel Young's modulus E[N] (dtype RVE_F32/RVE_F64,
 * finite and >= 0, not all zero) and the Poisson ratio nu in (-1, 0.5)
 * (isotropic small-strain Hooke's law, Sec. 3.3; plane strain in 2D).
 * E = 0 is a zero-stiffness (vacuum) voxel (Sec. 3.2): the projected operator
 * is then only semi-definite and CG runs on its range.  The mean stresses,
 * C_eff and the strains of every element with E > 0 are unique (the energy is
 * strictly convex in them); strains of zero-stiffness elements, and the
 * adjoint gradient at zero-stiffness voxels, can carry any null-space
 * component and are not. */
int rve_set_material(rve_t h, const void* E, int E_dtype, double nu, int ptr_flags);

/* Solve L load cases together.  E_macro[L][n_s] (host, Mandel) are the
 * macroscopic strains (the k = 0 mode, Sec. 2.3).  rel_tol bounds the final
 * relative FP64 nodal residual ||B^T C (E + eps~)|| / ||B^T C E||; a load case
 * whose residual reaches the FP64 round-off level of its nodal-force sums
 * (64 eps times the norm of the summed term magnitudes) also counts as solved,
 * which covers macroscopic strains that are already in equilibrium; max_iter
 * bounds the projected-CG iterations of each load case.  info[L] (host,
 * may be NULL) receives per-load-case statistics.  Returns the worst status. */
int rve_solve(rve_t h, const double* E_macro, int L, double rel_tol, int max_iter,
              rve_info* info);

/* Mean stresses of the solved load cases: S[L][n_s] (host, FP64), the volume
 * average of C : (E_l + eps~_l) over all elements. */
int rve_mean_stress(rve_t h, double* S);

/* Effective tangent C_eff[n_s][n_s] (host, FP64, Mandel, row-major) from the
 * last solve, which must have had L = n_s linearly independent load cases:
 * the matrix with C_eff E_macro[l] = S[l] for every l, i.e.
 * C_eff = S^T M^-T with M[l][:] = E_macro[l]. */
int rve_effective_tangent(rve_t h, double* C);

/* Energy form of the homogenised stiffness for the solved load cases:
 * Ce[a][b] = mean over all elements of (E_a + eps~_a) : C : (E_b + eps~_b)
 * (host, FP64, L x L, row-major).  At the exact solution it equals
 * E_a . C_eff E_b; its error is second order in the solve error, which makes it
 * the quantity to difference in finite-difference checks. */
int rve_energy_tangent(rve_t h, double* Ce);

/* Adjoint gradient of J = sum_ab W[a][b] C_eff[a][b] with respect to the
 * per-voxel Young's moduli, grad_E[N] (FP64).  Needs a preceding solve with
 * L = n_s independent load cases.  For every row a of W that is not zero it
 * runs the adjoint projected-CG solve (same operator, right-hand side -G C e_a)
 * and then forms
 *   dJ/dE_v = 1/(N n_q) sum_{Theta in v} sum_{a,l} W'[a][l]
 *             (e_a + lambda_a)_Theta : Cbar : eps_l,Theta,    W' = W M^-1. */
int rve_adjoint(rve_t h, const double* W, double rel_tol, int max_iter,
                void* grad_E, int ptr_flags);

/* Total strain field of a solved load case, eps[m][N] in FP64 (E + eps~). */
int rve_get_strain(rve_t h, int load_case, void* eps, int ptr_flags);

/* One application of the projected operator q = G * (C : p) to a field
 * p[m][N] (dtype of the handle's inner precision: RVE_F64 for RVE_FP64,
 * RVE_F32 for RVE_MIXED), written to q[m][N].  With apply_material = 0 the
 * material step is skipped and q = G * p (the bare projection). */
int rve_apply_operator(rve_t h, const void* p, void* q, int apply_material, int ptr_flags);

/* Schedule of the FFT passes: tile shapes, threads and radix schedules.
 * variants[RVE_SCHED_PASSES] holds
 *  [0] the first pass (material + x FFT): 0 default rows per block, 1 half,
 *      2 double; with n_x >= 64 also 3 default rows and 4 half rows with one
 *      thread per 16-byte load unit of the tile; in 3D with RVE_MIXED and
 *      n_x >= 128 also 5, a persistent pipelined pass whose next tile's rows
 *      arrive by bulk copies while the current tile is transformed (CG
 *      iterations of up to 64 load cases; otherwise it runs as 0), and 6,
 *      variant 0 whose blocks each ask for a later block's rows to be
 *      prefetched into L2 (a hint: no wait, same arithmetic).  A bounded
 *      device-side wait of variant 5 that gives up makes the solve return
 *      RVE_ERR_TIMEOUT.  In 2D with RVE_MIXED and n_x = 512 or 1024, 5 is the
 *      x transform with each 32-point register FFT spread over a pair of
 *      lanes (fewer registers, three blocks per SM);
 *  [1] the last pass (inverse x FFT + CG update): 0 default rows, 1 half, 2 double;
 *      in 3D with RVE_MIXED and n_x >= 128 also 3, a persistent pipelined
 *      pass whose next spectrum tile arrives by one tensor copy (same
 *      conditions and timeout as variant 5 of the first pass), and 4, variant
 *      0 with the L2 prefetch of a later block's spectrum tile and rows;
 *  [2] the split N = N1 * N2 of the four-step FFT along the last axis (y in
 *      2D, z in 3D; the pass that applies the projection): 0 the most square
 *      split, 1 half N1 and twice N2 (16 = 2 x 8, 32 = 2 x 16, 64 = 4 x 16,
 *      128 = 4 x 32, 256 = 8 x 32; lengths 512 and 1024 have only split 0);
 *  [3] in 3D the same choice for the y transforms (0 or 1); 0 in 2D.
 * -1 = choose by timing the candidates on the handle's buffers at the next
 * solve, with that solve's load cases (at most 8) (the default; the choice is
 * cached per grid, precision and number of load cases timed for the
 * process).  rve_set_schedule rejects a variant the grid does not have.
 * rve_schedule also returns the measured candidate times
 * candidate_ms[RVE_SCHED_PASSES][RVE_SCHED_VARIANTS] (0 where a candidate does
 * not exist or was not timed; may be NULL). */
enum { RVE_SCHED_PASSES = 4, RVE_SCHED_VARIANTS = 7 };
int rve_schedule(rve_t h, int* variants, float* candidate_ms);
int rve_set_schedule(rve_t h, const int* variants);

/* Order of the projected operator inside the CG iterations.  Both forms apply
 * the same operator G C (Eq. stat-mech-equi-FFT-homogenization with the
 * projection of Eqs. discrete_projection_op and small-strain-eq2), so the CG
 * iterates agree up to rounding:
 *   RVE_FORM_STRESS   (default) forward FFT of every stress component, the
 *                     projection B (B^H B)^-1 B^H at each wavevector, inverse
 *                     FFT of every strain component.
 *   RVE_FORM_FACTORED the same chain split where Appendix B splits it: the
 *                     right-hand side of Eq. small-strain-eq2 (B^H applied to
 *                     the stresses) is formed in real space as nodal forces
 *                     with the element stencils of Eq. discrderiv, only the D
 *                     nodal components are FFT'd and multiplied by the
 *                     inverse normal matrix (B^H B)^-1 (Eq. small-strain-chi),
 *                     and the strains of Eq. small-strain are formed back in
 *                     real space with the same stencils.  It needs one more
 *                     direction field [L][m][N] of the inner precision.
 *   RVE_FORM_NODAL    the factored chain with the CG vectors themselves kept
 *                     as nodal fields: every iterate of the projected CG is
 *                     compatible, x = B xi, r = B rho, p = B pi, so CG runs on
 *                     D components per node (xi, rho, pi) with the inner
 *                     products taken in strain space (<B pi, C B pi>,
 *                     |B rho|^2) and the same alpha, beta, stopping test and
 *                     iterates in exact arithmetic; the strain field is
 *                     recovered as E + B u.  This is the reading of the
 *                     projection as a preconditioner of the FE stiffness that
 *                     Sec. 4 points to.  No extra memory.
 * rve_set_operator_form applies from the next solve; returns RVE_ERR_ARG for
 * an unknown form, RVE_ERR_OOM if the extra field cannot be allocated. */
#define RVE_FORM_STRESS 0
#define RVE_FORM_FACTORED 1
#define RVE_FORM_NODAL 2
int rve_set_operator_form(rve_t h, int form);
int rve_operator_form(rve_t h, int* form);

/* Discrete derivative of the projection (B(k) and n_q, the evaluation points
 * per voxel).  RVE_DERIV_FE (default) is the linear-finite-element projection
 * (Sec. 2.6: two triangles / six Kuhn tetrahedra per voxel).  The others are
 * the comparison operators of the paper, one evaluation point per voxel unless
 * stated:
 *   RVE_DERIV_FOURIER   i k (Eq. original-G; on even grids the Nyquist
 *                       component of k is taken as 0, the average of the two
 *                       grid choices of Sec. 2.7),
 *   RVE_DERIV_CENTRAL   central differences (Eq. central-difference-derivative-fourier),
 *   RVE_DERIV_FORWARD   forward differences (Eq. forward-difference-derivative-fourier),
 *   RVE_DERIV_LSQ       the least-squares voxel gradient of Sec. 2.5,
 *   RVE_DERIV_FOURIER2  the Fourier derivative at the two triangle centroids
 *                       (Appendix C; 2D only, n_q = 2).
 * G = 0 wherever every symbol vanishes (k = 0; for central differences, least
 * squares and the Fourier derivative also some Nyquist wavevectors).  The
 * non-FE derivatives have no nodal real-space residual, so their solve is the
 * plain projected CG on the strain fluctuation in FP64 (the handle must be
 * RVE_FP64 and in RVE_FORM_STRESS; otherwise RVE_ERR_ARG), stopping on
 * ||r|| <= rel_tol ||r0||; rve_adjoint and rve_energy_tangent are for
 * RVE_DERIV_FE only.  Changing the derivative drops the handle's solution
 * and per-load-case buffers (the strain field then has m = n_q n_s
 * components; rve_sizes reports it); rve_apply_operator uses the handle's
 * derivative.  rve_derivative returns the code and n_q (nq may be NULL). */
#define RVE_DERIV_FE 0
#define RVE_DERIV_FOURIER 1
#define RVE_DERIV_CENTRAL 2
#define RVE_DERIV_FORWARD 3
#define RVE_DERIV_LSQ 4
#define RVE_DERIV_FOURIER2 5
int rve_set_derivative(rve_t h, int derivative);
int rve_derivative(rve_t h, int* derivative, int* nq);

/* ---- Finite strain ----------------------------------------------------
 * rve_set_kinematics(h, RVE_FINITE_STRAIN) switches the handle to
 * deformation gradients: the unknown per element is F = F_macro + H with
 * F_ia = d chi_i / d r_a (Eq. def-grad), compatibility by the projection of
 * Eq. original-G built from the element derivatives (G_iabj = delta_ij g_ab,
 * g from Eq. discrete_projection_op), equilibrium G P(F) = 0 (Eq.
 * stat-mech-equi-FFT-homogenization) for the first Piola-Kirchhoff stress of
 * the St. Venant-Kirchhoff law (our reading of the "isotropic finite strain
 * linear elastic law" of Sec. 3.1): E = (F^T F - I)/2, S = lambda tr(E) I +
 * 2 mu E, P = F S, with lambda and mu from the voxel's modulus and the
 * Poisson ratio (plane strain in 2D).  The solve is Newton with each
 * correction from projected CG on the tangent (G K(F) G is self-adjoint).
 * Requirements: RVE_FP64, RVE_FORM_STRESS, RVE_DERIV_FE; in 3D n_z <= 128
 * (RVE_ERR_UNSUPPORTED_SIZE otherwise).  Switching drops the solution and
 * the per-load-case buffers; rve_solve and rve_adjoint are then refused
 * (RVE_ERR_ARG), rve_apply_operator applies the bare gradient projection
 * (apply_material = 0 only) to fields of m = 9 (2D: 2 x 4 + one zero
 * padding component) or 54 (3D) components, element major, F_ia at
 * element * D*D + i*D + a.
 *
 * rve_solve_finite: F_macro[L][D][D] (row-major F_ia, host), Newton stops when
 * ||G P(F)|| <= rel_tol ||G P(F_macro)|| or at the round-off level of |P|;
 * info[l].refine_steps counts Newton steps, .iterations CG iterations,
 * .rel_residual the final Newton residual, .status RVE_OK /
 * RVE_ERR_NOT_CONVERGED (max_newton or max_iter reached) / RVE_ERR_NONFINITE.
 * rve_mean_piola: P[L][D][D], the mean first Piola-Kirchhoff stress.
 * rve_get_deformation: F[n_q][D][D][N] (FP64) of one load case. */
#define RVE_SMALL_STRAIN 0
#define RVE_FINITE_STRAIN 1
int rve_set_kinematics(rve_t h, int kinematics);
int rve_solve_finite(rve_t h, const double* F_macro, int L, double rel_tol, int max_newton, int max_iter,
                     rve_info* info);
int rve_mean_piola(rve_t h, double* P);
int rve_get_deformation(rve_t h, int load_case, void* F, int ptr_flags);

/* Measurement hooks (not part of the method).  With timing enabled, every
 * kernel launch of the solver is bracketed by CUDA events on the handle's
 * stream; rve_timing_read returns, per kernel kind, the summed device time in
 * milliseconds and the number of launches since the last read, and resets
 * them.  Kinds (index), counting launches inside projected-CG iterations:
 * 0 pass A (material + x FFT; factored form: x FFT of the nodal forces),
 * 1 pass B (y FFT, 3D), 2 pass C (last-axis FFT + projection or nodal solve),
 * 3 pass D (inverse y FFT, 3D), 4 pass E (inverse x FFT + CG update; factored
 * form: inverse x FFT of w); 5 the FP64 residual; 6 every other launch
 * (right-hand side, displacement recovery, homogenisation); 7 the real-space
 * material kernel of the factored and nodal forms (force stencil / force
 * kernel) and of finite strain (direction update and tangent); 8 the
 * real-space update kernel of the factored and nodal forms.  Kind 5 also
 * counts the finite-strain stress evaluations of the Newton residual. */
#define RVE_NKINDS 9
int rve_timing_enable(rve_t h, int enable);
int rve_timing_read(rve_t h, double* ms /*[RVE_NKINDS]*/, int64_t* launches /*[RVE_NKINDS]*/);

/* ---- Batches of RVEs of uneven grid size -------------------------------
 * A batch holds `count` RVEs of one dimension and precision, each with its own
 * grid (same size rules as rve_create) and per-voxel moduli, and one Poisson
 * ratio.  RVEs of equal grid size form a group whose RVEs x load cases are
 * solved together as batch slots of one set of launches (every slot has its own
 * CG scalars and stops on its own); the groups run concurrently on streams of
 * their own.  The batch owns all device memory; calls return after the work is
 * done. */
typedef struct rve_batch_s* rve_batch_t;

/* n[count * dim] grid sizes (x first per RVE). */
int rve_batch_create(rve_batch_t* out, int dim, int count, const int64_t* n, int precision, double nu);
int rve_batch_destroy(rve_batch_t b);
/* Moduli of RVE `index` (same rules as rve_set_material). */
int rve_batch_set_material(rve_batch_t b, int index, const void* E, int E_dtype, int ptr_flags);
/* Solve the L load cases E_macro[L][n_s] for every RVE; info[count][L] (may be
 * NULL).  Returns the worst status over all slots. */
int rve_batch_solve(rve_batch_t b, const double* E_macro, int L, double rel_tol, int max_iter, rve_info* info);
/* Mean stresses S[L][n_s] / effective tangent C[n_s][n_s] (L = n_s) of RVE `index`. */
int rve_batch_mean_stress(rve_batch_t b, int index, double* S);
int rve_batch_effective_tangent(rve_batch_t b, int index, double* C);

/* Allocation-free operator application (the paper has no counterpart; this is
 * a service for callers that cannot allocate device memory, e.g. code inside
 * an application that owns the whole device memory pool through its own
 * allocator, or latency-critical loops where an allocation may block or fail).
 * Computes q = G * (C : p) (apply_material = 1) or q = G * p (0) for a 2D grid
 * in FP32, like rve_apply_operator on an RVE_MIXED handle, without a handle and
 * without calling cudaMalloc/cudaFree or any allocating routine.
 *  n[2]       grid sizes, powers of two with 16 <= n <= 256; larger grids
 *             return RVE_ERR_SCRATCH_LIMIT;
 *  length[2]  cell lengths (NULL = unit cell);
 *  E[N]       device pointer, FP32 Young's moduli (may be NULL if apply_material = 0);
 *  p, q       device pointers, [6][N] FP32 fields (layout as rve_get_strain);
 *  cuda_stream  stream to run on (NULL = default stream).
 * Scratch: one static device array of about 1.6 MB (spectrum, tables and a
 * state record), which every GPU that loads the library holds until the process
 * exits.  That memory is taken when the library's device code is loaded on a
 * device: with lazy module loading (the CUDA default) this happens at the first
 * call on that device (or at the first use of any other entry point there), so
 * a caller that must not allocate later makes one call at set-up time.  The
 * first call on a device also looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make that first call before
 * any stream capture.  Later calls copy nothing from the host: the tables and
 * the state record are written by a small kernel.  All calls share the array
 * and it keeps the contents of the last call (each call rewrites everything it
 * reads), so calls that overlap on the GPU -- on different streams, or from
 * different host threads -- race; serialise them.  Not usable after
 * cudaDeviceReset on that device.  Returns without waiting for the GPU. */
int rve_apply_operator_2d_static(const int64_t* n, const double* length, const float* E, double nu,
                                 const float* p, float* q, int apply_material, void* cuda_stream);

/* Test hook (the paper has no counterpart): with on != 0 the pipelined passes
 * (schedule variant 5 of the first pass, 3 of the last) issue none of their
 * copies, so that their bounded device-side waits run out; the solve then
 * returns RVE_ERR_TIMEOUT after a few seconds and the handle stays usable once
 * the hook is off again.  For testing the timeout path without a GPU fault;
 * off by default, no effect on other schedules. */
int rve_test_stall_copies(rve_t h, int on);

/* Number of voxels N and strain scalars per voxel m of a handle. */
int rve_sizes(rve_t h, int64_t* n_voxels, int* m, int* n_s, int* dim);

#ifdef __cplusplus
}
#endif
#endif /* RVE_H */
