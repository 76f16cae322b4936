/*
 * pie.h -- C ABI of the GB300 library for the MLFMA matrix-vector product of
 * the potential integral equations (PIEs) of Guer & Erguel (2017).
 *
 * The operator is the Galerkin matrix Z of Eqs. (1)-(2) (Section 2): J on RWG
 * functions (one per interior edge) and sigma = n'.A on pulse functions (one
 * per triangle), N = E + T.  With <a,g,b> = int int a(r).b(r') g dr' dr and
 * g = exp(i k0 R)/(4 pi R):
 *
 *     Z_JJ[m,n] = mu0 <f_m, g, f_n>        Z_Js[m,t] = <div f_m, g, p_t>
 *     Z_sJ[t,n] = <p_t, g, div' f_n>       Z_ss[t,u] = w^2 eps0 <p_t, g, p_u>
 *
 * (Eq. (1) tested tangentially with the RWG functions, Eq. (2) with the
 * pulses, the gradient of g moved onto the testing function by parts as
 * Section 3 describes).  Constants: mu0 = 4 pi 1e-7, c0 = 299792458,
 * eps0 = 1/(mu0 c0^2), w = k0 c0.  Unknowns and results are ordered
 * [E RWG coefficients ; T pulse coefficients]; edges are numbered in
 * increasing (min vertex, max vertex) order; the "+" triangle of an edge is
 * the one whose counter-clockwise vertex order runs along the edge from its
 * smaller to its larger vertex.
 *
 * The product splits (Section 3) into a near part -- exact pair integrals
 * between triangles in neighbouring leaf boxes of a cubic oct-tree
 * (one-box buffer) -- and a far part computed by aggregation, interpolation,
 * diagonal translation with the approximate stable diagonalization of
 * Eqs. (4)-(5), anterpolation and disaggregation.
 *
 * Conventions for every call:
 *  - Return value: PIE_OK or an error code; pie_last_error() gives a message
 *    (thread-local, valid until the next call on the same thread).  No call
 *    throws or aborts.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is enqueued on it asynchronously unless stated.
 *  - Complex arrays are interleaved (re, im) pairs: PIE_C128 = two doubles,
 *    PIE_C64 = two floats.
 *  - The library owns all memory it allocates; objects are not thread-safe.
 */
#ifndef PIE_H
#define PIE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PIE_OK = 0,
  PIE_ERR_PARAM = 1,        /* invalid argument */
  PIE_ERR_NONMANIFOLD = 2,  /* an edge is shared by more than two triangles */
  PIE_ERR_DEGENERATE = 3,   /* a triangle has zero area or repeated vertices */
  PIE_ERR_ORIENTATION = 4,  /* two triangles traverse a shared edge the same way */
  PIE_ERR_OOM = 5,          /* device or host allocation failed */
  PIE_ERR_CUDA = 6,         /* a CUDA runtime call failed */
  PIE_ERR_LEAF = 7,         /* leaf box smaller than 1.5 x the longest edge */
  PIE_ERR_NOCONV = 8,       /* GMRES did not reach the tolerance */
  PIE_ERR_BREAKDOWN = 9,    /* GMRES Arnoldi breakdown */
  PIE_ERR_NAN = 10          /* NaN or Inf met in the iteration */
} pie_status;

typedef enum { PIE_C128 = 0, PIE_C64 = 1 } pie_dtype;

/* Arithmetic of the product:
 *  PIE_FP64  everything in complex double (inputs/outputs PIE_C128);
 *  PIE_FP32  near and far parts in complex float (inputs/outputs PIE_C64);
 *  PIE_MIXED near part in complex float (pair moments stored as float),
 *            far part in complex double (inputs/outputs PIE_C128);
 *  PIE_FP32H as PIE_FP32, with the near pair moments stored in IEEE half
 *            precision, each of the eight moment planes scaled by its own
 *            power of two (largest magnitude in [2^14, 2^15)), stored
 *            pair by pair (one 32-byte record per pair) and converted
 *            back to float in the product: half the near-part bytes, a
 *            fixed relative rounding of ~2.4e-4 per moment.  Meant for the
 *            inner operator of pie_solve_nested.
 * Setup (pair integrals, translation operators, filters) is always FP64. */
typedef enum { PIE_FP64 = 0, PIE_FP32 = 1, PIE_MIXED = 2, PIE_FP32H = 3 } pie_precision;

typedef struct pie_mesh pie_mesh;
typedef struct pie_problem pie_problem;

typedef struct {
  int levels;        /* L >= 3; level 1 is the root box, translations at 3..L */
  double root_side;  /* side of the root cube in metres; <= 0: largest
                        bounding-box extent.  The cube is centred on the
                        vertex bounding-box centre. */
  int tau;           /* truncation number of Eq. (5) */
  double kappa_a;    /* x = (k0 / s_l) a_l, the same at every level, so the
                        scale factor of Eq. (4) is s_l = k0 a_l / x */
  int ntheta;        /* angular samples: ntheta (even) Gauss-Legendre nodes
                        in cos(theta) x 2 ntheta azimuths, P = 2 ntheta^2 */
  int precision;     /* pie_precision */
  int max_nrhs;      /* right-hand sides one pass of pie_apply handles (the
                        near part reads each pair's moments once for up to 8
                        of them); work buffers scale with it */
} pie_params;

typedef struct {
  int64_t N, E, T;            /* unknowns, RWG functions, triangles */
  int32_t L, P;               /* levels, angular samples per box */
  int64_t boxes[24];          /* occupied boxes per level, index = level */
  int64_t near_pairs;         /* triangle pairs in the near part */
  int64_t device_bytes;       /* device memory held by the problem */
  double leaf_size;           /* leaf box side in metres */
} pie_info;

typedef struct {
  int32_t iterations;         /* Arnoldi steps taken */
  double rel_residual;        /* ||b - Z x|| / ||b||, recomputed in FP64 */
  double seconds;             /* wall time of the solve */
  int32_t reorthogonalizations; /* Arnoldi steps that took a second Gram-Schmidt pass */
  double product_seconds;     /* part of `seconds` in operator products (CUDA events) */
} pie_solve_stats;

/* Message of the last failed call on this thread ("" if none). */
const char* pie_last_error(void);

/* Default parameters: levels 3, root_side 0, tau 7, kappa_a 0.08, ntheta 8,
 * precision PIE_FP64, max_nrhs 1: product error below 1e-3 with an FP64 rounding
 * nonlinearity (~2.5e-6) low enough for GMRES to reach 1e-6 (the error and
 * rounding trade-off of Eqs. (4)-(5)). */
void pie_params_default(pie_params* p);

/* Surface mesh (Section 2: triangulated surface S).  xyz: nv x 3 doubles
 * (metres, host); tri: nt x 3 vertex indices (host, counter-clockwise seen
 * from the side the normal points to).  The library copies both arrays and
 * builds the RWG table.  Boundary edges (one triangle) carry no RWG, so open
 * surfaces are allowed.  Errors: PIE_ERR_PARAM (index out of range, nt = 0),
 * PIE_ERR_DEGENERATE, PIE_ERR_NONMANIFOLD, PIE_ERR_ORIENTATION. */
pie_status pie_mesh_create(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt,
                           pie_mesh** out);
void pie_mesh_destroy(pie_mesh* m);
/* Counts of the mesh (host values). */
pie_status pie_mesh_info(const pie_mesh* m, int64_t* nv, int64_t* nt, int64_t* ne);
/* Edge table (host arrays, E x 2 each): vertex pairs (min, max), triangles
 * (T+, T-), free vertices opposite the edge in (T+, T-).  Any pointer may be
 * NULL. */
pie_status pie_mesh_edges(const pie_mesh* m, int32_t* edges, int32_t* edge_tri, int32_t* edge_free);

/* Operator set-up for wavenumber k0 (rad/m): oct-tree and lists (host),
 * near pair integrals, radiation tables, translation operators of Eq. (5)
 * and interpolation filters (device kernels, FP64).  Synchronises the
 * stream before returning.  Errors: PIE_ERR_PARAM, PIE_ERR_LEAF, PIE_ERR_OOM,
 * PIE_ERR_CUDA. */
pie_status pie_problem_create(const pie_mesh* m, double k0, const pie_params* p, void* stream,
                              pie_problem** out);
void pie_problem_destroy(pie_problem* pr);
pie_status pie_problem_info(const pie_problem* pr, pie_info* info);

/* Tree export for bit-exact checks (host arrays).
 * pie_problem_perm: perm[T], the mesh triangle at each tree position
 *   (triangles sorted by (leaf Morton key, triangle index)).
 * pie_problem_level: for level l in [1, L]: keys[nb] (Morton keys, sorted);
 *   for l >= 3 also the interaction lists in CSR form: ptr[nb+1], idx[ptr[nb]]
 *   (source box numbers, ascending) and off[ptr[nb]] (offset code 0..315 of
 *   destination minus source box index, lexicographic over {-3..3}^3 without
 *   {-1..1}^3).  Call with NULL arrays to get nb and the list length.
 * pie_problem_near: leaf near lists, ptr[nleaf+1] and idx[...].  */
pie_status pie_problem_perm(const pie_problem* pr, int64_t* perm);
pie_status pie_problem_level(const pie_problem* pr, int level, int64_t* nb, int64_t* nlist,
                             int64_t* keys, int64_t* ptr, int64_t* idx, int32_t* off);
pie_status pie_problem_near(const pie_problem* pr, int64_t* nlist, int64_t* ptr, int64_t* idx);

/* y = Z x (Section 3: one MVM).  x, y: device buffers of N x nrhs complex
 * numbers, column-major (column j at offset j*N), caller-owned, not
 * overlapping; right-hand sides run in batches of max_nrhs.  dtype must be PIE_C128 for PIE_FP64 / PIE_MIXED problems and
 * PIE_C64 for PIE_FP32.  Asynchronous on the stream.  Errors: PIE_ERR_PARAM,
 * PIE_ERR_CUDA. */
pie_status pie_apply(pie_problem* pr, const void* x, void* y, int nrhs, int dtype, void* stream);

/* y = Z^T x (conj = 0) or y = Z^H x (conj = 1), same arguments and errors as
 * pie_apply.  The Galerkin operator of Eqs. (1)-(2) is complex symmetric
 * (reciprocity); the discrete one keeps that: the near pair moments are
 * two-sided, and the far part is symmetric on the antipodal angular grid
 * (aggregation and disaggregation are each other's transposes, anterpolation
 * is the transposed interpolation, T_{-w}(k) = T_w(-k)).  Z^T x therefore runs
 * the forward stages (equal to Z x up to the far part's rounding, ~1e-5), and
 * Z^H x = conj(Z conj x).  Uses one N-vector of library scratch. */
pie_status pie_apply_t(pie_problem* pr, const void* x, void* y, int nrhs, int dtype, int conj, void* stream);

/* y = Z_near x: the near part of the product alone (Section 3: interactions
 * of triangles in neighbouring leaf boxes, one-box buffer, computed exactly
 * as in the dense matrix).  Same arguments and errors as pie_apply.  Useful
 * as a sparse preconditioner and for checking the near part by itself. */
pie_status pie_apply_near(pie_problem* pr, const void* x, void* y, int nrhs, int dtype, void* stream);

/* The product split by where its interactions run (Section 3).  Every
 * triangle pair (t, s) -- boxes by centroid -- is either near (neighbouring
 * leaf boxes) or translated at exactly one level l in [3, L]: the level at
 * which the ancestor boxes of t and s stop being neighbours (their parents
 * are neighbours).  y = near * Z_near x + sum of Z_l x over the levels l
 * whose bit (1u << l) is set in level_mask; level_mask = 0xFFFFFFFF with
 * near = 1 is pie_apply, and the parts sum to it up to the far part's
 * rounding.  For per-level error checks against exact pair sums: after the
 * call, pie_problem_stage(pr, 3, ...) holds the per-triangle potentials of
 * the far part alone.  One right-hand side (x, y: device, N complex of the
 * problem's dtype).  Errors: PIE_ERR_PARAM, PIE_ERR_CUDA. */
pie_status pie_apply_levels(pie_problem* pr, const void* x, void* y, uint32_t level_mask, int near, int dtype,
                            void* stream);

/* Allocation-free variant of pie_apply_near (the paper has no counterpart:
 * this serves callers that cannot allocate device memory when they need a
 * product -- code inside a CUDA-graph capture they do not own, hosts that
 * forbid allocation after start-up, frameworks whose allocator owns all
 * device memory).  Computes y = Z_near x for one right-hand side (x, y:
 * device, N complex of the problem's dtype) and calls no cudaMalloc,
 * cudaFree or other allocating routine.  Its per-triangle scratch (local
 * coefficients and potentials, 2 x 6 complex per triangle) lives in one
 * fixed 24 MiB device array inside the library, which every GPU that loads
 * the library holds until the process exits; meshes above 131072 triangles
 * (complex double) or 262144 (complex float) are rejected with
 * PIE_ERR_PARAM.  The array's device address is looked up
 * (cudaGetSymbolAddress) by pie_problem_create, on the device current there,
 * and kept in the problem; so the entry point itself does no set-up and may
 * be called inside a stream capture, and it returns PIE_ERR_PARAM when the
 * current device is not the problem's.  All calls share the array and every
 * call overwrites the parts it reads, so nothing carries over between calls;
 * calls that overlap on the GPU (different streams, or different problems
 * at once) race on it.  Errors: PIE_ERR_PARAM, PIE_ERR_CUDA. */
pie_status pie_apply_near_noalloc(pie_problem* pr, const void* x, void* y, int dtype, void* stream);

/* Per-stage timing of products (CUDA events recorded on the apply stream
 * around each stage).  pie_profile_begin arms recording for the next
 * max_applies single-column products; pie_profile_end waits for them and
 * writes the summed milliseconds of the PIE_NSTAGES stages to stage_ms
 * (host, may be NULL) and the number of recorded products to applies.
 * Stages, in order: 0 local coefficients, 1 near part, 2 leaf aggregation,
 * 3 interpolation (all levels), 4 translation (all levels), 5 anterpolation,
 * 6 leaf disaggregation, 7 Galerkin assembly. */
#define PIE_NSTAGES 8
pie_status pie_profile_begin(pie_problem* pr, int max_applies);
pie_status pie_profile_end(pie_problem* pr, double* stage_ms, int32_t* applies);

/* Stage output of the last pie_apply (first right-hand side), copied to the
 * host after synchronising the stream: which = 0 radiated patterns S_l
 * (after aggregation / interpolation), which = 1 incoming patterns G_l (after
 * translation and anterpolation), 2 = per-triangle local coefficients
 * [T][6] (a, beta_x, beta_y, beta_z, sigma, d) in tree order (level ignored),
 * 3 = per-triangle potentials [T][6] (U, V_x, V_y, V_z, T1, T2) of the far
 * part (of the near part after pie_apply_near), 4 = near
 * pair moments [8][nnz] (m0, mt_xyz, ms_xyz, mts; entries ordered by test
 * triangle in tree order, then by near box, then by source triangle),
 * 5 = leaf radiation table Pi [T][P/2], 6 = leaf radiation table M
 * [T][3][P/2] (tree order; the half grid of theta rows 0..ntheta/2-1, the
 * other half being the complex conjugates at the antipodes).  Patterns
 * are [nb][5][P] complex double (converted from float in PIE_FP32). */
pie_status pie_problem_stage(pie_problem* pr, int which, int level, double* out, void* stream);

/* Right-hand side for a plane wave E = pol E0 exp(i k0 khat.r) (pol . khat =
 * 0) with the Lorenz-gauge potentials Phi = -E0 (pol.r) exp(i k0 khat.r),
 * A = -(E0/c0)(pol.r) khat exp(i k0 khat.r):  b_J = -<f_m, A>,
 * b_sigma = -i w eps0 <p_t, Phi> (Eqs. (1)-(2) right-hand sides).  b: device,
 * N complex of the problem's dtype. */
pie_status pie_rhs_planewave(pie_problem* pr, const double khat[3], const double pol[3], double E0,
                             void* b, int dtype, void* stream);

/* The problem's quadrature points (Section 2: the Galerkin integrals over
 * each triangle use a 7-point degree-5 rule): pts [T][7][3] and weights
 * (area included) wts [T][7], host, mesh order; either may be NULL.  Where
 * a caller evaluates its own incident potentials for pie_rhs_potentials. */
pie_status pie_problem_quadrature(const pie_problem* pr, double* pts, double* wts);

/* Right-hand side for any incident potentials (Eqs. (1)-(2)): A^inc and
 * Phi^inc given at the points of pie_problem_quadrature, A_q [T][7][3] and
 * Phi_q [T][7] (device, complex double, mesh order).  b_J = -<f_m, A^inc>,
 * b_sigma = -i w eps0 <p_t, Phi^inc>, with the same rule as the operator.
 * b: device, N complex of the problem's dtype.  Errors: PIE_ERR_PARAM. */
pie_status pie_rhs_potentials(pie_problem* pr, const void* A_q, const void* Phi_q, void* b, int dtype,
                              void* stream);

/* Far-zone field from J (Section 2): E[d] = i w mu0/(4 pi) (I - rr) .
 * int J exp(-i k0 r.r') dr' (factor exp(i k0 r)/r removed).  rhat: host
 * ndir x 3; x: device solutions, N x nrhs (problem dtype, column j at
 * offset j*N); E: device nrhs x ndir x 3 complex double. */
pie_status pie_farfield(pie_problem* pr, const void* x, const double* rhat, int64_t ndir, void* E, int nrhs,
                        void* stream);

/* Adjoint of the far-field map of pie_farfield: u = F^H E for E (device,
 * ndir x 3 complex double) at the host directions rhat (ndir x 3); u:
 * device, N complex of the problem's dtype (pulse entries are zero: the far
 * zone depends on J only, Section 2).  Used for gradients of far-field
 * objectives through an adjoint solve. */
pie_status pie_farfield_adjoint(pie_problem* pr, const double* rhat, int64_t ndir, const void* E, void* u,
                                void* stream);

/* GMRES (Section 4) on Z x = b, zero initial guess, restarted every
 * `restart` steps, stopping when the FP64 residual ||b - Z x||/||b|| <= tol
 * (the operator is scaled symmetrically by the inverse square roots of the
 * diagonal magnitudes of its near part; the stopping test is on the
 * unscaled system: a cycle ends when the rotated residual of the scaled
 * system falls to tol / 2 or the unscaled residual of the iterate, formed
 * from the Krylov basis every 4 steps, to tol, and the true residual
 * b - Z x then decides; after twelve cycles in a row so ended whose true
 * residual missed tol, later cycles run at least 25 steps, then 50, ...).  PIE_FP64 problems keep the Krylov basis in complex
 * double; PIE_MIXED problems keep it in complex float, with the solution and
 * the true residual in complex double recomputed at every restart (iterative
 * refinement with a GMRES inner solver), so the basis precision limits the
 * progress of a cycle, not the accuracy reached.  b, x: device, N x nrhs
 * complex double (column j at offset j*N), solved column after column;
 * stats: nrhs entries (host, may be NULL).  Synchronises the stream.
 * Returns PIE_OK when every column converged, else PIE_ERR_NOCONV or
 * PIE_ERR_BREAKDOWN of the first column that did not (the other columns are
 * still solved); PIE_ERR_PARAM (PIE_FP32 problem), PIE_ERR_NAN and
 * PIE_ERR_CUDA stop at once.  There is no wall-clock limit: maxit bounds
 * the work. */
pie_status pie_solve(pie_problem* pr, const void* b, void* x, int nrhs, double tol, int maxit, int restart,
                     pie_solve_stats* stats, void* stream);

/* pie_solve from the caller's x (N x nrhs, device, read as the initial
 * guess and overwritten with the solution): the first residual is
 * b - Z x instead of b.  Resumes an interrupted solve from a saved x (the
 * operator is rebuilt deterministically from mesh, k0 and parameters), or
 * starts a nearby right-hand side from a previous solution.  Same
 * arguments, stopping test and errors as pie_solve. */
pie_status pie_solve_guess(pie_problem* pr, const void* b, void* x, int nrhs, double tol, int maxit, int restart,
                           pie_solve_stats* stats, void* stream);

/* Nested mixed-precision solve of Z x = b (Section 4 solves with GMRES; the
 * inner operator is the same discrete PIE operator with its far part at an
 * Eqs. (4)-(5) point whose rounding amplification complex float tolerates).
 * Flexible GMRES (Saad 1993) on the outer problem's operator -- far part in
 * FP64 -- right-preconditioned by one GMRES cycle on the inner problem's
 * operator per outer step: z_j = (inner cycle from zero on v_j), product
 * Z z_j with the outer operator.  Both operators are scaled by the outer
 * problem's near-part diagonal (as pie_solve).  The outer Krylov vectors,
 * the solution and the true residual b - Z x (recomputed with the outer
 * operator at every outer restart) are complex double; the inner basis is
 * complex float unless the inner problem is PIE_FP64.
 *   outer: PIE_FP64 or PIE_MIXED problem; inner: any precision, built on the
 *     same mesh (identical vertex and triangle arrays) at the same k0 (its
 *     levels and (tau, kappa_a, ntheta) may differ);
 *   b, x: device, N x nrhs complex double (column j at offset j*N), solved
 *     column after column from x = 0;
 *   stats: nrhs entries (host, may be NULL).
 * Parameters (pie_nested_params):
 *   tol: stopping test ||b - Z x|| / ||b|| <= tol with the outer operator;
 *   maxit: bound on inner Arnoldi steps (inner products) per column;
 *   inner_restart: steps of one inner cycle (1..1000);
 *   inner_tol: an inner cycle stops once its residual has fallen by this
 *     factor (0 < inner_tol < 1);
 *   outer_restart: outer steps per restart (1..200); 0 = iterative
 *     refinement (x += D z for the preconditioned scaled residual);
 *   max_outer: bound on products with the outer operator per column.
 * Measured on GB300 (PIE_MIXED outer, PIE_FP32H inner at tau 3, kappa_a
 * 0.15, N_theta 4): inner_restart 20, inner_tol 0.05, outer_restart 80
 * reach 1e-6 in 1.6-1.9 s at 819,200 unknowns and in 52 s at 3,276,800;
 * shorter inner cycles were faster on some right-hand sides but needed up
 * to 5 times more outer products on others.
 * An outer cycle ends when its rotated (scaled) residual or the unscaled
 * residual of its iterate (formed from the outer Krylov basis every step)
 * reaches tol, or after outer_restart steps; the FP64 true residual then
 * decides (after twelve cycles in a row so ended whose true residual missed
 * tol, later cycles run at least 5 steps, then 10, ...).
 * Synchronises the stream.  Returns PIE_OK when every column converged, else
 * PIE_ERR_NOCONV of the first column that did not; PIE_ERR_PARAM (mismatched
 * problems, PIE_FP32 outer problem, parameters out of range), PIE_ERR_OOM,
 * PIE_ERR_NAN and PIE_ERR_CUDA stop at once. */
typedef struct {
  double tol;
  int32_t maxit;
  int32_t inner_restart;
  double inner_tol;
  int32_t outer_restart;
  int32_t max_outer;
} pie_nested_params;

typedef struct {
  int32_t inner_iterations;     /* inner Arnoldi steps (products with the inner operator) */
  int32_t outer_iterations;     /* outer steps (inner cycles) */
  int32_t outer_products;       /* products with the outer operator, true residuals included */
  double rel_residual;          /* ||b - Z x|| / ||b|| with the outer operator, FP64 */
  double seconds;               /* wall time of the solve */
  double inner_product_seconds; /* part of `seconds` in inner products (CUDA events) */
  double outer_product_seconds; /* part of `seconds` in outer products (CUDA events) */
} pie_nested_stats;

pie_status pie_solve_nested(pie_problem* outer, pie_problem* inner, const void* b, void* x, int nrhs,
                            const pie_nested_params* params, pie_nested_stats* stats, void* stream);

/* Near-zone fields (Section 2).  The far zone needs J only; near-zone E needs
 * the charge density rho = i w eps0 n'.A - eps0 n'.grad'Phi, whose second
 * term solves Eq. (3): int_S (n'.grad'Phi) g = Phi^inc on S (the total scalar
 * potential vanishes on the conductor).  Eq. (3) is discretised with the
 * pulses and tested with them, i.e. with the single-layer operator
 * S_tu = <p_t, g, p_u> -- the pulse-pulse block of Z divided by w^2 eps0 --
 * which runs through the same near and far stages as Z.
 * All vectors here are complex double, device, and need a PIE_FP64 or
 * PIE_MIXED problem; T-vectors are in mesh order.
 *
 * pie_apply_single_layer: y = S q (q, y: T complex).
 * pie_solve_single_layer: GMRES on S q = b, same stopping test, scaling
 *   (|S_tt|^-1/2) and error codes as pie_solve.
 * pie_rhs_potential: b_t = <p_t, Phi^inc> for the plane wave of
 *   pie_rhs_planewave (Phi^inc = -E0 (pol.r) exp(i k0 khat.r)).
 * pie_nearfield: scattered field E_s(r) = i w mu0 int J g - (1/eps0) int rho
 *   grad g at npts host points pts (npts x 3, off the surface; the 7-point
 *   rule per triangle is accurate beyond about one triangle size), from the
 *   PIE solution x (N) and the charge-density pulse coefficients rho (T).
 *   E: device npts x 3 complex double. */
pie_status pie_apply_single_layer(pie_problem* pr, const void* q, void* y, void* stream);
pie_status pie_solve_single_layer(pie_problem* pr, const void* b, void* x, double tol, int maxit, int restart,
                                  pie_solve_stats* stats, void* stream);
pie_status pie_rhs_potential(pie_problem* pr, const double khat[3], const double pol[3], double E0, void* b,
                             void* stream);
pie_status pie_nearfield(pie_problem* pr, const void* x, const void* rho, const double* pts, int64_t npts, void* E,
                         void* stream);

/* Launch choices of the product (the paper, one MATLAB process, has none;
 * they change where and how the stages run, never the arithmetic, so the
 * product is the same to the last bit under every setting).
 *  overlap: 1 = the near part (HBM-bound) runs on a second stream of the
 *    problem and the far part on a third one of the device's highest
 *    priority (on the caller's stream while that stream is being captured
 *    into a graph), forked from the caller's stream after the local
 *    coefficients and joined back before the assembly (the far part's short
 *    kernels take SM slots ahead of the near part's many blocks).
 *    0 = the caller's stream alone, stages in order.
 *  near_ctas_per_sm: grid of the near kernel when overlapped, in CTAs of 256
 *    threads per SM (each warp walks test triangles with a grid stride), so
 *    that it takes a bounded share of every SM beside the far kernels;
 *    0 = one warp per test triangle.  0..32.
 *  rhs_chunk: right-hand sides per pass over the operator, 1..max_nrhs.
 *  near_rhs_block: right-hand sides that one pass of the near kernel
 *    carries (each pair's moments are read once for them): 1, 2, 4 or 8
 *    (8 only with the warp-per-triangle kernel), or 0 to pick by the pass
 *    width (1 for one column, 2 for two or a complex double near part, 4 up
 *    to four, else 8).
 *  far_rows: tile shape of the per-box far kernels of angular grids other
 *    than N_theta = 8 (aggregation, dense interpolation and anterpolation,
 *    translation; one thread per sample): boxes per block, 1, 2, 4, 8, 16 or
 *    32, reduced where a block would exceed 1024 threads or 48 KB of shared
 *    memory; 0 = automatic (enough boxes to fill 128 threads).
 *  near_kernel: near-part kernel for a float near part: 1 = one warp per
 *    test triangle reading the coefficients from global memory (1, 2, 4 or
 *    8 right-hand sides per thread), 2 = box-staged (one block per leaf box
 *    and group of up to 4 right-hand sides, the box's source coefficients
 *    in shared memory), 0 = automatic (box-staged for passes of one column,
 *    warp per triangle otherwise).  Both take the same operations in the
 *    same order.  A complex double near part, and near_rhs_block 8, always
 *    use the warp-per-triangle kernel.
 * Defaults at pie_problem_create: overlap 1, near_ctas_per_sm 2, rhs_chunk
 * max_nrhs, near_rhs_block 0, far_rows 0, near_kernel 0.  Per-stage
 * profiling (pie_profile_begin) runs the stages in order whatever overlap
 * says. */
typedef struct pie_tuning {
  int32_t overlap;
  int32_t near_ctas_per_sm;
  int32_t rhs_chunk;
  int32_t near_rhs_block;
  int32_t far_rows;
  int32_t near_kernel;
} pie_tuning;

pie_status pie_problem_get_tuning(const pie_problem* pr, pie_tuning* t);
/* Errors: PIE_ERR_PARAM (a field out of range). */
pie_status pie_problem_set_tuning(pie_problem* pr, const pie_tuning* t);

/* Autotuner: times products of nrhs right-hand sides (1..1024; library
 * scratch, contents irrelevant to the timing) under each candidate setting
 * -- overlap off, overlap with near_ctas_per_sm in {1, 2, 3, 4, 6, 8, 0},
 * rhs_chunk in the powers of two up to min(nrhs, max_nrhs), near_rhs_block
 * in {1, 2, 4, 8} up to the chosen chunk, far_rows in {1, 2, 4, 8, 16} when
 * N_theta is not 8, near_kernel 1 and 2 for a float near part -- by CUDA events
 * on the stream, median of reps (1..100) after one warm-up each, keeps the
 * fastest, and returns it (best, host) with its
 * milliseconds per right-hand side (best_ms, host, may be NULL).  The search
 * is greedy: the overlap grid at the largest rhs_chunk first, then
 * rhs_chunk, then near_rhs_block, then far_rows, then near_kernel.  Allocates
 * 2 x nrhs x N complex of scratch for its duration; synchronises the stream.
 * Errors: PIE_ERR_PARAM, PIE_ERR_OOM, PIE_ERR_CUDA. */
pie_status pie_problem_autotune(pie_problem* pr, int nrhs, int reps, pie_tuning* best, double* best_ms,
                                void* stream);

/* Level count per mesh: builds the problem of mesh m at k0 with base's other
 * parameters for every L in [lmin, lmax] whose leaf box admits the mesh
 * (leaf side >= 1.5 x the longest edge; others are skipped), autotunes each
 * for nrhs right-hand sides, and returns the L with the fewest milliseconds
 * per right-hand side (best_levels, host).  ms_per_level (host, may be NULL)
 * receives lmax - lmin + 1 entries, 0 where L was skipped.  The product's
 * accuracy does not depend on L at fixed (tau, kappa_a, ntheta).  Each
 * candidate is set up and destroyed in turn (peak memory: one problem).
 * Errors: PIE_ERR_PARAM, PIE_ERR_LEAF (no admissible L), the set-up errors. */
pie_status pie_tune_levels(const pie_mesh* m, double k0, const pie_params* base, int lmin, int lmax, int nrhs,
                           void* stream, int* best_levels, double* ms_per_level);

/* Arithmetic peaks of the current device for the roofline of the ALU-bound
 * kernels (the paper has no counterpart: a measurement aid).  Times fused
 * multiply-add chains (eight independent chains per thread, the chain value
 * either the multiplicand or the addend, 4 or 8 blocks of 256 threads per
 * SM: the best of the four forms) in real FP64 and FP32 with CUDA events on
 * the stream, best of three launches after ten untimed ones, about 2 s in all;
 * writes TFLOP/s (2 flop per FMA) and the SM clock in MHz that the best
 * launch ran at (clock64 ticks over globaltimer nanoseconds: long FMA
 * streams can run below the maximum clock under the power limit) to the
 * host doubles.  Synchronises the stream.  Errors: PIE_ERR_PARAM (NULL
 * output), PIE_ERR_CUDA. */
pie_status pie_measure_peaks(double* fp64_tflops, double* fp32_tflops, double* fp64_mhz, double* fp32_mhz,
                             void* stream);

/* Multi-mesh batch: several problems (meshes of uneven size, any
 * wavenumbers and precisions) applied to nrhs right-hand sides each in ONE
 * launch.  pie_group_apply captures, on first use of a given set of
 * buffers, the products of all members into one CUDA graph -- each member on
 * its own branch, so that the small stages of one mesh fill the SMs left
 * idle by another -- and launches that graph on the stream; later calls
 * with the same (x, y, nrhs) relaunch it (the graphs of the four most recent
 * buffer sets are kept).  x[i], y[i]: device buffers of member i, N_i x nrhs
 * complex in that member's dtype (PIE_C64 for PIE_FP32 problems, PIE_C128
 * otherwise), column-major as in pie_apply.  Members keep their own state:
 * a member must not be applied by other calls while a group launch that
 * holds it may run, nor destroyed before the group; profiling must be off.
 * pie_group_info: graphs captured so far and group launches (host, may be
 * NULL).  Errors: PIE_ERR_PARAM (n < 1, NULL member or buffer, nrhs out of
 * range, a member profiling), PIE_ERR_CUDA. */
typedef struct pie_group pie_group;
pie_status pie_group_create(pie_problem* const* members, int n, pie_group** out);
pie_status pie_group_apply(pie_group* g, const void* const* x, void* const* y, int nrhs, void* stream);
pie_status pie_group_info(const pie_group* g, int64_t* graphs, int64_t* launches);
void pie_group_destroy(pie_group* g);

#ifdef __cplusplus
}
#endif
#endif /* PIE_H */
