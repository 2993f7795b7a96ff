/*
 * tpp.h - C ABI of libtpp: approximate tensor-product (Kronecker SVD)
 * preconditioned, matrix-free GMRES for very-high-order DG advection on GB300.
 *
 * Method: W. Pazner and P.-O. Persson, "Approximate tensor-product
 * preconditioners for very high order discontinuous Galerkin methods".
 *
 * Problem (Sec. 3.4, Sec. 5.1 Eq. adv): linear advection u_t + div(a u) = 0 on a
 * periodic Cartesian mesh of nel[0] x nel[1] (x nel[2]) elements of width h,
 * n = p + 1 Gauss-Legendre nodes per direction, quadrature collocated with the
 * nodes, upwind numerical flux.  One implicit step gives the system
 *     S x = (M - dt J) x = (M + dt A) x = b,        A = -J.
 *
 * Data layout of every solution-sized vector (device, float64): element-major,
 * element e = ex + nel[0] * (ey + nel[1] * ez), and inside an element the DOF
 * index i + n j (+ n^2 k) with x fastest.  Kronecker factors act as
 * A (x) B (2D: A on y, B on x) and A (x) B (x) C (3D: z, y, x).
 *
 * Conventions shared by all entry points:
 *  - Every pointer argument documented as "device" must point to memory on the
 *    current CUDA device; "host" pointers are read before the call returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls enqueue work on it and return without synchronising, except where a
 *    host-side report is filled (tpp_create, tpp_build_factors, gmres_solve).
 *  - The library never allocates device memory: all device state lives in the
 *    caller's workspace (size from tpp_workspace_bytes), owned by the caller and
 *    valid for the lifetime of the context.
 *  - Errors: a non-zero tpp_status is returned and a message is available from
 *    tpp_last_error() (thread-local).  Device kernels never trap; failures they
 *    detect are written to status words and reported by the next reporting call.
 *  - There is no CPU fallback: without a usable GB300 device every call fails
 *    with TPP_ERR_CUDA.
 */
#ifndef TPP_H
#define TPP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TPP_OK = 0,
  TPP_ERR_INVALID_ARG = 1,     /* bad size, null pointer, aliasing, option out of range */
  TPP_ERR_CUDA = 2,            /* a CUDA runtime call failed (message has the CUDA error) */
  TPP_ERR_SINGULAR_FACTOR = 3, /* an inverted Kronecker factor is numerically singular */
  TPP_ERR_NOT_CONVERGED = 4,   /* GMRES hit max_iters before rtol */
  TPP_ERR_BREAKDOWN = 5,       /* Arnoldi breakdown before convergence */
  TPP_ERR_SCHUR = 6,           /* Francis QR did not converge within its iteration cap */
  TPP_ERR_NAN = 7,             /* NaN or Inf met in a residual */
  TPP_ERR_UNSUPPORTED = 8,     /* valid request this build does not implement */
  TPP_ERR_WORKSPACE = 9,       /* workspace too small or misaligned */
  TPP_ERR_TIMEOUT = 10         /* a device-side pipeline wait gave up (status word set; no trap) */
} tpp_status;

/* Arithmetic of the Kronecker apply: FP64; FP32 (float factors and arithmetic); BF16
 * (BF16 factors and stage inputs, FP32 accumulation, on the tensor cores; 2D, n <= 16,
 * contexts with TPP_FEAT_BF16). */
typedef enum { TPP_FP64 = 0, TPP_FP32 = 1, TPP_BF16 = 2 } tpp_prec;

typedef enum {
  TPP_PC_NONE = 0,         /* unpreconditioned */
  TPP_PC_KRON = 1,         /* KSVD Kronecker preconditioner (Alg. 2d-apply / 3d-apply) */
  TPP_PC_BLOCK_JACOBI = 2  /* exact block Jacobi (dense LU of each diagonal block) */
} tpp_pc;

/* Feature bits for tpp_workspace_bytes / tpp_create. */
#define TPP_FEAT_BLOCK_JACOBI 1u  /* reserve n^(2d) doubles per element for exact block Jacobi */
#define TPP_FEAT_MIXED        2u  /* reserve float32 copies of the Kronecker apply factors */
#define TPP_FEAT_TWO_SIDED    4u  /* apply by the paper's two-sided Schur form (quasi-triangular
                                     Sylvester solve) instead of the default one-sided form */
#define TPP_FEAT_LEARNED      8u  /* reserve the buffers of tpp_build_factors_learned (2D) */
#define TPP_FEAT_TIME        16u  /* reserve 6 solution-sized vectors for tpp_time_integrate */
#define TPP_FEAT_BF16        32u  /* reserve BF16 copies of the apply factors for TPP_BF16
                                     (2D, n <= 16, one-sided form) */
#define TPP_FEAT_F32_SHIFTS 128u  /* with TPP_FEAT_MIXED (one-sided form, n <= 16, mu <= n): the
                                     build forms the shifted inverses of the one-sided form in
                                     FP32 only, for the FP32 apply (no 2 n^3 doubles per
                                     element); Kronecker applies are then TPP_FP32 only */
#define TPP_FEAT_FULL_BLOCKS 64u  /* system contexts (tpp_create_system): Kronecker factors
                                     (2D, n <= 16; 3D nested form) and, with
                                     TPP_FEAT_BLOCK_JACOBI, exact LU (2D, n <= 16; 3D, n <= 6)
                                     of the whole n_c n^d element blocks instead of the n_c
                                     small ones (Sec. 5.3, 5.6) */

/*
 * Problem description (Sec. 3.4, Sec. 5.1 Eq. adv): the system S x = (M + dt A) x = b of
 * one implicit step of u_t + div(a u) = 0, discretised on num_elem elements of width h
 * (squares / cubes of side h, affine), n = p + 1 Gauss-Legendre nodes per direction,
 * quadrature collocated with the nodes, upwind flux.  The library needs the flux
 * Jacobians of Alg. matrix-free-matvec (steps 1-2): dF_c/du = a_c at the volume nodes and
 * a . n_outward at the face nodes, given here as arrays, and the element connectivity.
 *
 *  vel_nodes        device [dim][num_elem * n^dim]: a_c at the volume nodes, element-major,
 *                   node index i + n j (+ n^2 k), x fastest.
 *  vel_face_normal  device [num_elem][2 dim][n^(dim-1)]: a . n_outward at the face nodes,
 *                   faces ordered -x, +x, -y, +y (, -z, +z), face nodes by their tangential
 *                   indices in (x, y, z) order, the first fastest.  Both sides of an interior
 *                   face should carry opposite values (the caller's data is used as given).
 *  nbr              device [num_elem][2 dim]: the element across each face, which meets it
 *                   with its opposite face (-x against +x, ...) and the same tangential node
 *                   order; -1 for no coupling (the face keeps only its own outflow term, so a
 *                   problem with every entry -1 is a batch of block-diagonal systems).
 * The three arrays are read by tpp_create (and tpp_set_velocity) only; the library keeps
 * its own copies.  nrhs right-hand sides per element are stored together in every vector:
 * layout [num_elem][nrhs][n^dim] (float64 unless stated).
 * Limits: dim in {2, 3}; 1 <= n <= 32 (2D), 1 <= n <= 16 (3D); num_elem >= 1; nrhs >= 1;
 * h > 0; dt >= 0; every nbr entry in [-1, num_elem).
 *
 * Over-integration (mu > n, Sec. 3.2 with the mu-point Gauss-Legendre rule, 2D): the
 * integrals of the operator are evaluated at mu points per direction (the evaluation and
 * derivative matrices G and D of the nodal basis at the quadrature points, Table
 * tab:dg-ops), so vel_nodes holds a at the mu^2 quadrature points of every element and
 * vel_face_normal a.n at the mu face quadrature points of every face (same orderings, mu in
 * place of n; tpp_gauss_legendre returns the rule).  The rearranged block then has rank up
 * to 2 mu + 2 instead of 2 n + 2 (the structure of Sec. 4.2.1 changes) and the factor
 * build works on the explicit core described at tpp_build_factors.  Not with
 * TPP_FEAT_BLOCK_JACOBI or TPP_FEAT_LEARNED.
 */
typedef struct {
  int32_t dim;
  int32_t n;
  int64_t num_elem;
  int32_t nrhs;
  int32_t mu;          /* quadrature points per direction: 0 or n = collocated with the nodes;
                          n < mu <= 32 = over-integration (2D), see below */
  double h;
  double dt;
  const double* vel_nodes;
  const double* vel_face_normal;
  const int32_t* nbr;
} tpp_problem;

typedef struct {
  int32_t restart;      /* GMRES(m) restart length, 1 <= m <= max_restart of the context */
  int32_t max_iters;    /* total Arnoldi steps over all cycles, >= 1 */
  double rtol;          /* stop when ||b - A x|| <= rtol ||b||, rtol > 0 */
  int32_t pc;           /* tpp_pc */
  int32_t inner_prec;   /* tpp_prec of the Kronecker apply; TPP_FP32 needs TPP_FEAT_MIXED,
                           TPP_BF16 TPP_FEAT_BF16 (and TPP_FEAT_MIXED for inner solves) */
  int32_t flexible;     /* 1: flexible GMRES (stores Z = P^-1 V); forced to 1 when inner_prec != FP64 */
  int32_t inner_iters;  /* 0: each preconditioner application is one Kronecker apply.  k > 0
                           (mixed precision, needs TPP_FEAT_MIXED and TPP_PC_KRON): it is an
                           inner FP32 GMRES solve S d = v of at most k steps (k <= max_restart),
                           right-preconditioned by the FP32 Kronecker apply, with the FP32
                           operator and FP32 basis vectors; the outer solve is flexible GMRES
                           in FP64 (operator, Arnoldi, Givens, true residual). */
  int32_t use_graph;    /* 1: every group of Arnoldi steps between two host reads of the solver
                           state (8 steps; 1 outer step when inner_iters > 0) runs as one CUDA
                           graph, captured at its first use and kept in the context for later
                           cycles and solves with the same restart, pc, inner_prec, flexible,
                           inner_iters and inner_rtol (another combination recaptures); a group
                           cut short by max_iters runs as plain launches.  Same kernels in the
                           same order as 0, so the same iterates.  0 or 1. */
  double inner_rtol;    /* inner solves stop early at this relative residual estimate (0: never) */
} tpp_gmres_opts;

typedef struct {
  int32_t iters;        /* Arnoldi steps taken */
  int32_t cycles;       /* restart cycles */
  int32_t status;       /* tpp_status of the solve */
  int32_t converged;    /* 1 when the true relative residual <= rtol */
  double true_rel_res;  /* ||b - A x|| / ||b|| of the returned x */
  double est_rel_res;   /* last Arnoldi (Givens) estimate */
  int32_t inner_iters;  /* total inner FP32 steps (inner_iters > 0 in the options) */
  int32_t reserved;
} tpp_gmres_result;

typedef struct {
  int32_t num_elem;
  int32_t num_shifted;     /* elements that inverted A2 + alpha A1 and B1 - alpha B2 with
                              alpha != 0 (same P; chosen for conditioning) */
  int32_t num_rank1;       /* elements with sigma_2 <= 1e-14 sigma_1 (P = A1 (x) B1) */
  int32_t num_schur_fail;  /* elements whose Francis iteration hit its cap */
  double max_cond;         /* largest cond_1(L_A) * cond_1(L_B) of the inverted factor pair */
  double min_sigma_ratio;  /* min over elements of sigma_2 / sigma_1 */
  double max_cond_z;       /* 3D: largest cond_1(A1) of the first-stage z factor (0 in 2D) */
  int32_t num_z_unconverged;  /* 3D: elements whose first-stage Lanczos hit its step cap
                                 (the factor is still the best Ritz pair found) */
  int32_t num_fallback;     /* tpp_build_factors_learned: elements given the exact KSVD */
  int32_t num_schur_relaxed;  /* elements whose Francis iteration deflated a nearly defective
                                 eigenvalue cluster at sqrt(eps) instead of eps (flags bit 4):
                                 their factors are those of a matrix within sqrt(eps) |C| */
} tpp_build_report;

typedef struct tpp_ctx tpp_ctx;

/*
 * Bytes of device workspace a context needs (256-byte aligned start required).
 * max_restart bounds the GMRES restart length later requested; features is a
 * mask of TPP_FEAT_*.  Returns 0 when the problem is invalid.
 */
size_t tpp_workspace_bytes(const tpp_problem* prob, int32_t max_restart, uint32_t features);

/*
 * Create a context on the caller's workspace and run the precomputation step of
 * Alg. matrix-free-matvec (steps 1-2): 1D Gauss-Legendre tables, the flux
 * Jacobians dF/du = a at volume nodes and a.n at face nodes scaled by the
 * quadrature weights (Sec. 3.4.1), the connectivity, and the element-independent
 * basis of the rearranged block used by the factor build.  vel_nodes and
 * vel_face_normal may be NULL (a zero field, to be set by tpp_set_velocity before
 * the first build); nbr may not.  Synchronises `stream` before returning.
 * workspace: device, ws_bytes >= tpp_workspace_bytes(prob, max_restart, features).
 */
tpp_status tpp_create(tpp_ctx** out, const tpp_problem* prob, int32_t max_restart,
                      uint32_t features, void* workspace, size_t ws_bytes, void* stream);

/* Release the host-side context (the workspace stays the caller's). */
void tpp_destroy(tpp_ctx* ctx);

/*
 * Replace the linearisation data of a context (Alg. matrix-free-matvec steps 1-2 again):
 * the velocity at the nodes and faces (layouts as in tpp_problem; device, read before
 * the call returns) and the step dt >= 0.  The factors and block-Jacobi LU of the old
 * operator become stale: call tpp_build_factors (and tpp_build_block_jacobi) again.
 * Synchronises `stream`.
 */
tpp_status tpp_set_velocity(tpp_ctx* ctx, const double* vel_nodes, const double* vel_face_normal,
                            double dt, void* stream);

/* Points and weights of the context's quadrature rule on [0, 1] (host arrays of mu
 * doubles: the n Gauss-Legendre nodes when collocated, the mu-point rule when
 * over-integrated), for callers that evaluate their field at the quadrature points.
 * Synchronises the legacy stream. */
tpp_status tpp_gauss_legendre(const tpp_ctx* ctx, double* nodes, double* weights);

/*
 * Form the Kronecker preconditioner of every element (Alg. 2d-form in 2D,
 * Alg. 3d-form in 3D): best rank-2 (3D: nested rank-1 then rank-2) Kronecker
 * approximation of the exact diagonal block by a Golub-Kahan-Lanczos SVD of its
 * Van Loan-Pitsianis rearrangement (Sec. 4.1, Alg. lanczos), LU inverses of the
 * factors the paper inverts (L_A, L_B), and the factor products C1 = L_A^-1 A1,
 * C2 = L_B^-1 B2.  With TPP_FEAT_TWO_SIDED: real Schur forms of C1 and C2
 * (Eq. quad-triang, as in the paper).  Default (one-sided form): the real Schur
 * form C1 = Q1 T1 Q1^T only, and for every 1x1 / 2x2 diagonal block J of T1 the
 * inverse of the shifted system I (x) C2 + T1[J, J] (x) I (Gauss-Jordan, partial
 * pivoting); the same P, stored in 2 n^3 extra doubles per element.
 * 2D: the inverted pair is (A2 + alpha A1, B1 - alpha B2),
 * which leaves P = A1 (x) B1 + A2 (x) B2 unchanged; alpha = 0 is the paper's
 * choice and a nonzero alpha is taken only when it lowers the condition
 * numbers of the inverted factors.  Factors are stored in the workspace.  `report` (host, may
 * be NULL) is filled after a stream synchronisation.
 * Returns TPP_ERR_SINGULAR_FACTOR / TPP_ERR_SCHUR when an element could not be
 * factored (the report counts them).
 * Over-integrated problems (mu > n): with the element-independent basis B = [vec(g_b g_b^T) |
 * vec(d_b g_b^T) | vec(l1 l1^T) | vec(l0 l0^T)] (g_b, d_b the rows of G and D at quadrature
 * point b, l0 / l1 the endpoint values) the rearranged block is A~ = B K B^T with K built
 * from the element's weights and flux Jacobians at the quadrature points; one Householder
 * QR B = Q R per context gives A~ = Q (R K R^T) Q^T, and the top-2 triplets come from the
 * dense SVD of the small core R K R^T (size min(n^2, 2 mu + 2)), O(mu^3) per element.
 */
tpp_status tpp_build_factors(tpp_ctx* ctx, tpp_build_report* report, void* stream);

/*
 * Exact block-Jacobi comparator: assemble each n^d x n^d diagonal block from the
 * flux Jacobians and LU-factor it (dense, partial pivoting).  Needs
 * TPP_FEAT_BLOCK_JACOBI.  Asynchronous.
 */
tpp_status tpp_build_block_jacobi(tpp_ctx* ctx, void* stream);

/*
 * x = P^-1 b, element by element (Alg. 2d-apply / 3d-apply).  P^-1 b is
 * (C1 (x) I + I (x) C2)^-1 (L_A^-1 (x) L_B^-1) b, i.e. X solves C2 X + X C1^T =
 * L_B^-1 B L_A^-T (B[i, j] = b[i + n j]).  Two-sided form: b~ = S_B B S_A^T,
 * quasi-triangular Sylvester solve T2 Y + Y T1^T = b~, x = Q2 Y Q1^T.  One-sided
 * form (default): R = L_B^-1 B S_A^T, then C2 Z + Z T1^T = R column block by
 * column block from the last with the stored shifted inverses, x = Z Q1^T.
 * 3D applies the A1^-1 factor along z first, then the 2D form on each z slice.
 * b, x: device float64 [num_elem][nrhs][n^dim], 1 <= nrhs <= the problem's nrhs, must not
 * alias.  prec selects the arithmetic and factor precision (TPP_FP32 needs
 * TPP_FEAT_MIXED; TPP_BF16 needs TPP_FEAT_BF16: one CTA per element, the three dense
 * stages and the column sweep as BF16 tensor-core products with FP32 accumulation, eight
 * right-hand sides per warp).  Asynchronous.
 */
tpp_status tpp_apply_inverse(const tpp_ctx* ctx, const double* b, double* x, int32_t nrhs,
                             int32_t prec, void* stream);

/* x = (block-Jacobi)^-1 b with the exact block LU factors (layout and nrhs as in
 * tpp_apply_inverse).  Asynchronous. */
tpp_status tpp_apply_block_jacobi(const tpp_ctx* ctx, const double* b, double* x, int32_t nrhs,
                                  void* stream);

/*
 * y = (M + dt A) x by sum factorisation (Alg. matrix-free-matvec step 3): mass
 * h^d w(x)w, volume -dt h^(d-1) sum_c (D^T along c) of w a_c x, upwind face
 * fluxes lifted by the endpoint values; across a face with neighbour e' the
 * inflow reads the same right-hand side r of e'.  x, y: device float64
 * [num_elem][nrhs][n^dim], 1 <= nrhs <= the problem's nrhs, must not alias.
 * Asynchronous.
 */
tpp_status dg_apply_sumfact(const tpp_ctx* ctx, const double* x, double* y, int32_t nrhs,
                            void* stream);

/*
 * FP32 forms used by the inner solves of the mixed-precision mode (contexts
 * created with TPP_FEAT_MIXED): the same operator on float vectors with float
 * copies of the flux Jacobian coefficients (FP32 arithmetic throughout), and
 * x = P^-1 b with the FP32 factors on float vectors (tpp_apply_inverse_f32
 * needs tpp_build_factors first).  Vectors: device float32 [num_elem][nrhs][n^dim],
 * must not alias.  The paper has no FP32 variant; these follow Sec. 3.4 and Alg.
 * 2d-apply / 3d-apply in single precision.  Asynchronous.
 */
tpp_status dg_apply_sumfact_f32(const tpp_ctx* ctx, const float* x, float* y, int32_t nrhs,
                                void* stream);
tpp_status tpp_apply_inverse_f32(const tpp_ctx* ctx, const float* b, float* x, int32_t nrhs,
                                 void* stream);

/*
 * Solve S x = b by restarted right-preconditioned GMRES(m) (Sec. 5 opening;
 * classical Gram-Schmidt with one reorthogonalisation, Givens rotations on
 * the device).  b: device float64 [num_dofs]; x: device float64 [num_dofs],
 * on entry the initial guess, on exit the solution.  The problem's nrhs
 * right-hand sides form one block-diagonal system (one Krylov space, residual
 * norms over all of them).  Synchronises `stream` and fills `result` (host,
 * required).
 */
tpp_status gmres_solve(tpp_ctx* ctx, const double* b, double* x, const tpp_gmres_opts* opts,
                       tpp_gmres_result* result, void* stream);

/*
 * Curved (non-affine) 2D elements: the general-geometry form of Sec. 3.2 (Eq. mass-kron,
 * adv-kron with a full element Jacobian J_T = dx/dxi at every quadrature point; the
 * paper's unstructured and curved meshes of Sec. 5.1).  The caller gives, at the
 * quadrature points of the context's rule (the n nodes, or the mu-point rule when
 * over-integrated; tpp_gauss_legendre), the metric terms folded with the velocity:
 *   jdet      device [E][q^2]      |J_T|                       (point a + q b, x fastest)
 *   flux      device [2][E][q^2]   F~ = |J_T| J_T^-1 a          (contravariant velocity)
 *   flux_face device [E][4][q]     a . (|J_T| J_T^-T N^)         (own side of faces -x, +x,
 *                                  -y, +y; N^ the reference outward normal)
 * For an affine element of width h these are h^2, h a and h a . n.  The mass becomes
 * w |J_T| point by point (applied through the mu-point rule when over-integrated), and
 * the factor build, block Jacobi and time integration use it.  Replaces the
 * coefficients of tpp_set_velocity (which returns the context to affine elements);
 * the factors must be rebuilt.  2D scalar contexts without TPP_FEAT_LEARNED
 * (TPP_ERR_UNSUPPORTED otherwise); not accepted by tpp_batch_gmres.  Synchronises
 * `stream`.
 */
tpp_status tpp_set_metric_terms(tpp_ctx* ctx, const double* jdet, const double* flux,
                                const double* flux_face, double dt, void* stream);

/*
 * Coupled systems of conservation laws (Sec. 5.3, Sec. 5.6: the Euler equations,
 * n_c = dim + 2 components rho, the momenta, rho E with the flux of Eq. euler-flux),
 * linearised around a DG state u0 given at the nodes.  The operator is the Jacobian
 * system S = M - dt J of the DG discretisation with the local Lax-Friedrichs flux
 * F^(u-, u+).n = 1/2 (F(u-) + F(u+)).n + 1/2 lam (u- - u+), lam = max(|v-.n| + c-,
 * |v+.n| + c+) frozen at u0: volume coefficients A_x(u0), A_y(u0) (n_c x n_c per node),
 * face coefficients 1/2 (A_n(u0-) + lam I) on the own trace and 1/2 (A_n(u0+) - lam I)
 * on the neighbour's.  By default the preconditioners are the paper's "small" ones:
 * the n_c diagonal n^d x n^d sub-blocks of every element block (no coupling between
 * components), approximated by the rank-2 Kronecker sum (K_small, nested in 3D) or
 * inverted exactly (block Jacobi, J_small).  With TPP_FEAT_FULL_BLOCKS they are the
 * "full" ones: in 2D (n <= 16) the whole n_c n^2 block approximated by A_1 (x) B_1 +
 * A_2 (x) B_2 with A_k of size n_c n on the (component, y) index and B_k of size n on
 * x (K_full), or inverted exactly (J_full, with TPP_FEAT_BLOCK_JACOBI); in 3D the nested
 * form A_1 (x) (B_1 (x) C_1 + B_2 (x) C_2) with A_1 of size n_c n on the (component, z)
 * index (first stage by power iteration, flagged in fflags bit0 if it has not converged
 * in 500 steps) and B_k, C_k of size n on y, x (K_full), or J_full (n <= 6).
 *
 * tpp_create_system returns an ordinary context whose elements are the (element,
 * component) pairs e * n_c + c: vectors are [E][n_c][n^dim], tpp_num_elem() is
 * E * n_c, dg_apply_sumfact / dg_apply_sumfact_static apply the coupled S, gmres_solve
 * solves with it, and tpp_build_factors / tpp_apply_inverse / tpp_build_block_jacobi
 * / tpp_apply_block_jacobi act on the small (or full) blocks.  Features:
 * TPP_FEAT_TWO_SIDED, TPP_FEAT_BLOCK_JACOBI, TPP_FEAT_BF16, TPP_FEAT_FULL_BLOCKS
 * (alone or with TPP_FEAT_BLOCK_JACOBI; others: TPP_ERR_INVALID_ARG).  tpp_set_velocity
 * must not be called on a system context (it would replace the small blocks only).
 */
#define TPP_FLUX_EULER 1
typedef struct {
  int32_t dim;              /* 2 or 3 */
  int32_t n;                /* nodes per direction, 1..32 (2D), 1..12 (3D) */
  int64_t num_elem;         /* physical elements E */
  int32_t nc;               /* components: dim + 2 for TPP_FLUX_EULER */
  int32_t flux;             /* TPP_FLUX_EULER */
  double gamma;             /* ratio of specific heats, > 1 (1.4 in the paper) */
  double h, dt;             /* element width (square elements), time step */
  const double* state;      /* device [E][nc][n^dim]: u0 in conserved variables (rho, the
                               momenta, rho E) at the nodes (read during tpp_create_system) */
  const int32_t* nbr;       /* [E][2 dim] neighbour across faces -x, +x, -y, +y (, -z, +z)
                               (-1: none), as in tpp_problem (read during tpp_create_system) */
} tpp_sys_problem;

/* Workspace for a system context (0 if invalid).  max_restart >= 5 and
 * (max_restart + 1) n >= dim (n + 2). */
size_t tpp_sys_workspace_bytes(const tpp_sys_problem* prob, int32_t max_restart,
                               uint32_t features);
/* As tpp_create; computes the linearisation coefficients from the state (synchronises
 * `stream`).  The workspace must hold tpp_sys_workspace_bytes. */
tpp_status tpp_create_system(tpp_ctx** out, const tpp_sys_problem* prob, int32_t max_restart,
                             uint32_t features, void* workspace, size_t ws_bytes, void* stream);

/*
 * Per-system batched GMRES over batches of isolated elements (an extension for
 * mixed-degree batches; each system is one element's diagonal block of Sec. 3.4,
 * S_e x = b with mass, volume and outflow face terms, solved by the
 * right-preconditioned restarted GMRES of Sec. 5 with the Kronecker preconditioner
 * of Alg. 2d-apply / 3d-apply).  Unlike gmres_solve, every (element, right-hand
 * side) system runs its own Arnoldi process with its own Givens rotations,
 * restarts and convergence test: ||b - S_e x|| <= rtol ||b|| per system.
 *
 * The contexts (one per degree group: dim, n) must be isolated (every nbr entry
 * -1), collocated (mu <= n), created with TPP_FEAT_TWO_SIDED (the two-sided factors
 * are staged in shared memory), with n <= 32 (2D) / n <= 16 (3D), factors built,
 * all on the current device; prec = TPP_FP32 also needs TPP_FEAT_MIXED.  The
 * systems run in persistent launches grouped by n (8, 16 or 32 lanes per system,
 * lane i owning row i of the n x n matrix of a vector or of its z slices); CTAs
 * take elements from one queue per launch, most expensive degree first, stage an
 * element's factors and flux coefficients in shared memory and solve its nrhs
 * systems warp by warp.
 *
 * prec TPP_FP64: GMRES(restart) in FP64.  prec TPP_FP32: FP64 iterative refinement
 * (true residual with the FP64 operator, up to max_outer steps) around FP32
 * GMRES(restart) solves of the correction to the relative residual inner_rtol
 * (FP32 operator, factors and Arnoldi vectors; Hessenberg and Givens in FP64).
 * max_iters bounds the Arnoldi steps of a system (summed over the inner solves).
 */
typedef struct {
  int32_t restart;          /* m, 1..31 */
  int32_t max_iters;        /* >= 1 */
  double rtol;              /* > 0 */
  int32_t prec;             /* TPP_FP64 or TPP_FP32 (mixed) */
  int32_t max_outer;        /* mixed: refinement steps (>= 1) */
  double inner_rtol;        /* mixed: relative tolerance of each FP32 solve, in (0, 1) */
  int32_t warps[3];         /* warps per CTA of the 8-, 16- and 32-lane launches, 1..8; 0: 8 */
  int32_t ctas_per_sm[3];   /* CTAs per SM of those launches; 0: as many as fit */
  int32_t reg_budget[3];    /* kernel variant of those launches: 1 = up to 255 registers per
                               thread, 2 = up to 128 (two 256-thread CTAs per SM); 0: 2 for
                               the 8- and 16-lane launches, 1 for the 32-lane one */
  int32_t* const* iters;    /* optional (NULL): per context a device int32 [E * nrhs] of
                               Arnoldi steps per system */
  double* const* relres;    /* optional (NULL): per context a device float64 [E * nrhs] of
                               final true relative residuals */
} tpp_batch_opts;

typedef struct {
  int64_t systems;          /* (element, right-hand side) systems solved */
  int64_t total_iters;      /* Arnoldi steps summed over the systems */
  int32_t max_iters;        /* largest per system */
  int32_t unconverged;      /* systems above rtol at exit */
  int32_t max_outer;        /* mixed: largest number of refinement steps */
  int32_t launches;         /* persistent launches made (one per lane-group width used) */
  double max_relres;        /* largest final true relative residual */
  double launch_ms[3];      /* device time of the 8-, 16- and 32-lane launches (0: none) */
} tpp_batch_report;

/* Workspace for tpp_batch_gmres with these contexts and options (0 if invalid;
 * tpp_last_error says why).  Queries the current device. */
size_t tpp_batch_workspace_bytes(tpp_ctx* const* ctxs, int32_t nctx, const tpp_batch_opts* opts);

/* ctxs: host array of nctx contexts; b, x: host arrays of nctx device float64
 * pointers [E][nrhs][n^d] (x overwritten, zero initial guess); workspace: device,
 * 256-byte aligned, ws_bytes >= tpp_batch_workspace_bytes, owned by the caller.
 * Synchronises `stream` and fills `report` (host, required).  Returns
 * TPP_ERR_INVALID_ARG for a context or option outside the limits above,
 * TPP_ERR_WORKSPACE for a small or misaligned workspace, TPP_ERR_NOT_CONVERGED if a
 * system ends above rtol (x still holds every system's last iterate). */
tpp_status tpp_batch_gmres(tpp_ctx* const* ctxs, int32_t nctx, const double* const* b,
                           double* const* x, const tpp_batch_opts* opts,
                           tpp_batch_report* report, void* workspace, size_t ws_bytes,
                           void* stream);

/*
 * dg_apply_sumfact_static: the same y = (M + dt A) x as dg_apply_sumfact, for
 * callers that cannot allocate device memory themselves (their device memory is
 * handed out by an allocator they do not control, or fixed once at start-up) and
 * so cannot provide scratch beyond the vectors they pass.  The face-trace scratch
 * lives in a static 4 MiB device array inside libtpp (held by every GPU that
 * loads the library until exit) instead of the context workspace; no device
 * memory is allocated.  The paper has no counterpart to this entry point.
 * x, y: device float64 [num_elem][nrhs][n^2], must not alias.  2D contexts with
 * num_elem * nrhs * 4 * n <= 524288 only; larger ones return TPP_ERR_INVALID_ARG.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array: calls that overlap on the GPU race.  The current device
 * must be the one the context was created on (TPP_ERR_INVALID_ARG otherwise), since
 * the array's address is that of the current device.  Asynchronous.
 */
tpp_status dg_apply_sumfact_static(const tpp_ctx* ctx, const double* x, double* y, int32_t nrhs,
                                   void* stream);

/*
 * Time integration of the semi-discrete system M u' = J u (Sec. 3.3, Eq. mass-u-r, with
 * the linear flux of Sec. 5.1; the context's operator is S = M - dt_ctx J, dt_ctx its
 * problem's dt).  Schemes:
 *  TPP_TS_BACKWARD_EULER  (M - dt J) u^{n+1} = M u^n  (the single implicit steps of Sec. 5.3-5.6);
 *  TPP_TS_DIRK3           the three-stage, third-order, L-stable DIRK method of Alexander used in
 *                         Sec. 5.2: stage values solve (M - gamma dt J) U_i = M (u^n + dt
 *                         sum_{j<i} a_ij k_j), k_i = M^-1 J U_i, u^{n+1} = U_3 (stiffly accurate);
 *  TPP_TS_RK4             the classical explicit fourth-order Runge-Kutta method (the explicit
 *                         comparison of Sec. 5.2); M is diagonal (collocated quadrature).
 * Implicit schemes first rescale the context's operator to dt_ctx = a_ii dt (dt for backward
 * Euler, gamma dt for DIRK3) when it differs (needs dt_ctx > 0; the context keeps the new dt),
 * build the Kronecker factors once, or before every step when rebuild_each_step (the paper's
 * setting, where the Jacobian changes every step), and solve every stage with gmres_solve and
 * `opts` (initial guess: the stage's explicit part).  RK4 applies J as -(S - M) / dt_ctx
 * through the operator without its mass term (needs dt_ctx > 0).
 * u: device float64 [num_dofs]: on entry u^0, on exit u after `steps` steps of size dt > 0.
 * Needs TPP_FEAT_TIME.  Synchronises `stream`; report (host, may be NULL) counts GMRES
 * iterations, factor builds and the largest true relative residual of any stage solve.
 * Returns the first failing solve's status (the integration stops there).
 */
typedef enum { TPP_TS_BACKWARD_EULER = 0, TPP_TS_DIRK3 = 1, TPP_TS_RK4 = 2 } tpp_time_scheme;
typedef struct {
  int32_t steps;            /* steps completed */
  int32_t gmres_iters;      /* Arnoldi steps over every stage solve */
  int32_t builds;           /* factor builds */
  int32_t solves;           /* stage solves */
  double max_true_rel_res;  /* largest ||b - S U|| / ||b|| of the stage solves */
} tpp_time_report;

tpp_status tpp_time_integrate(tpp_ctx* ctx, double* u, int32_t scheme, double dt, int32_t steps,
                              int32_t rebuild_each_step, const tpp_gmres_opts* opts,
                              tpp_time_report* report, void* stream);

/*
 * Element-wise inversion of the exact mass matrix (Sec. 3.3, Eq. mass-kron):
 *   M_K = (G^T W (x) ... (x) G^T W) J_T (G (x) ... (x) G)
 * with the mu-point Gauss-Legendre rule per direction (n <= mu <= 64; G the mu x n
 * evaluation matrix of the nodal basis at its points, W its weights) and J_T the
 * |Jacobian determinant| of each element's map at those points (curved or non-affine
 * elements), solved element by element by preconditioned conjugate gradients from x = 0
 * with the under-integrated (n-point, collocated) mass matrix as preconditioner: diagonal,
 * w (x) ... (x) w times J_T at the nodes (Sec. 3.3).  Stops at ||r|| <= rtol ||b|| per block.
 *  jac_q  device [num_elem][mu^dim]: |J_T| at the quadrature points (x fastest), including
 *         the element size (h^dim for an affine cube of side h);
 *  jac_n  device [num_elem][n^dim]: |J_T| at the nodes;
 *  r, x   device [num_elem][nrhs][n^dim] (must not alias);
 *  iters  device [num_elem * nrhs] iterations per block, or NULL.
 * Shared memory of one element block must fit 200 KB (2D: n <= 32, mu <= 64; 3D: e.g.
 * n <= 11 with mu <= 16), else TPP_ERR_UNSUPPORTED.  Synchronises `stream`; returns
 * TPP_ERR_NOT_CONVERGED when a block reached max_iters (x still written).
 */
tpp_status tpp_mass_solve(const tpp_ctx* ctx, int32_t mu, const double* jac_q,
                          const double* jac_n, const double* r, double* x, int32_t nrhs,
                          double rtol, int32_t max_iters, int32_t* iters, void* stream);

/* Device pointers into the workspace for inspection (tests); NULL if absent. */
typedef struct {
  const double* sigma;   /* [E][2] top singular values of the rearranged block (2D) */
  const double* A1;      /* [E][n*n] column-major factors, A on y (2D) */
  const double* B1;
  const double* A2;
  const double* B2;
  const double* SA;      /* [E][n*n] Q1^T L_A^-1 */
  const double* SB;      /* [E][n*n] Q2^T L_B^-1 (two-sided form); L_B^-1 (one-sided form) */
  const double* Q1;
  const double* Q2;      /* two-sided form only (NULL otherwise) */
  const double* T1;      /* real Schur form of C1 */
  const double* T2;      /* two-sided: real Schur form of C2; one-sided: C2 itself */
  const int32_t* flags;  /* [E] bit0 shifted pair, bit1 rank-1, bit2 schur fail, bit3 singular,
                            bit4 Schur deflated at sqrt(eps) */
  const double* cond;    /* [E] cond_1(L_A) * cond_1(L_B) of the inverted factor pair */
  const double* gl_x;    /* [n] Gauss-Legendre nodes on [0, 1] */
  const double* gl_w;    /* [n] weights */
  const double* D;       /* [n*n] D[a*n + j] = phi_j'(x_a) */
  /* 3D only (NULL in 2D).  The nested form A1 (x) (B1 (x) C1 + B2 (x) C2): the
   * second-stage factors of the y-x block D1 sit in A1/B1/A2/B2 above with A on
   * y and B on x, i.e. A1 = B1(3D), B1 = C1(3D), A2 = B2(3D), B2 = C2(3D); sigma
   * then holds the top two singular values of D1's rearrangement. */
  const double* Az;      /* [E][n*n] first-stage z factor A1 (3D), column-major */
  const double* Azi;     /* [E][n*n] its inverse */
  const double* sigz;    /* [E] first-stage singular value sigma_1 */
  const int32_t* zflags; /* [E] bit0 Lanczos not converged, bit1 A1 singular or cond_1 >= 1e14 */
  const double* G;       /* one-sided form: [E][n][2][n*n] shifted inverses Gs_j, Gp_j
                            (column-major n x n), NULL in the two-sided form */
  /* Over-integrated 2D contexts only (mu > n; NULL otherwise), r = tpp_core_size:
   * the rearranged block is A~ = Qb core Qb^T with B = Qb Rb (see tpp_build_factors) */
  const double* core;    /* [E][r*r] explicit cores R K R^T, column-major */
  const double* Qb;      /* [n^2 * r] orthonormal basis, column-major */
  const double* Rb;      /* [r][2 mu + 2] triangular factor of the basis B, row-major */
  const double* qtr;     /* [r] trace of mat(Qb[:, t]) */
  /* System contexts with TPP_FEAT_FULL_BLOCKS only (NULL otherwise), m = n_c n: the
   * factors of the whole element blocks, A_k on (component, y), B_k on x, row-major */
  const double* fA;      /* 2D: [E_phys][2][m][m] A_1, A_2; 3D: [E_phys][m][m] A_1 (the y-x
                            factors of the nested form sit in A1/B1/A2/B2 above, first
                            E_phys entries, with sigma their singular values) */
  const double* fB;      /* 2D: [E_phys][2][n][n]; NULL in 3D */
  const double* fsig;    /* [E_phys][2] 2D: sigma_1, sigma_2 of the rearranged block; 3D:
                            sigma_1 of the first stage, power iterations taken */
  const int32_t* fflags; /* [E_phys] bit0 first stage not converged (3D), bit1 rank-1, bit2
                            Schur fail, bit3 singular, bit4 relaxed */
} tpp_views;

tpp_status tpp_get_views(const tpp_ctx* ctx, tpp_views* out);

/* Stream-ordered device-to-device copy of `bytes` bytes (for callers that read
 * the views above without a CUDA runtime of their own).  Asynchronous. */
tpp_status tpp_copy_device(void* dst, const void* src, size_t bytes, void* stream);

/*
 * Learned Kronecker factors (an extension; the paper has no learned component).
 * A multilayer perceptron maps an element's velocity samples to its rank-2 factors:
 * 2 n^2 + 1 inputs (a_x and a_y at the n x n nodes, x fastest, then dt / h), three
 * hidden layers of width 512 with the exact GELU, 4 n^2 outputs read as vec(A_1),
 * vec(B_1), vec(A_2), vec(B_2) (column-major) of the rearranged block divided by its
 * Frobenius norm.  Parameters: FP32 master copies used as BF16 weights, FP32
 * accumulation everywhere.  Loss of an element: || A~/||A~|| - sum_k vec(A_k)
 * vec(B_k)^T ||_F^2 (gauge invariant; Sec. 4.1 Eq. NKP), evaluated through the
 * element's core M (A~ = Q M Q^T); the batch loss is the mean.  Training: Adam
 * (0.9, 0.999, 1e-8).  The network lives in a caller workspace like a context.
 */
typedef struct tpp_mlp tpp_mlp;
int64_t tpp_mlp_num_params(int32_t n);                      /* -1 for a bad n */
size_t tpp_mlp_workspace_bytes(int32_t n, int32_t max_batch);
tpp_status tpp_mlp_create(tpp_mlp** out, int32_t n, int32_t max_batch, void* workspace,
                          size_t ws_bytes, void* stream);
void tpp_mlp_destroy(tpp_mlp* net);
/* host params, FP32: for each layer l = 0..3, W_l [K_l][N_l] row-major, then b_l [N_l];
 * setting them resets the optimiser state */
tpp_status tpp_mlp_set_params(tpp_mlp* net, const float* host_params, void* stream);
tpp_status tpp_mlp_get_params(const tpp_mlp* net, float* host_params, void* stream);
/* X: device [B][2 n^2 + 1]; out: device [B][4 n^2]; 1 <= B <= max_batch */
tpp_status tpp_mlp_forward(tpp_mlp* net, const float* X, int32_t B, float* out, void* stream);
/* Forward, loss and gradients of a batch; with lr > 0 one Adam step.  Mn: device
 * [B][r*r] normalised cores from tpp_learned_inputs of `basis` (a 2D context of the
 * same n, whose structure basis defines Q); loss: device float, the batch mean. */
tpp_status tpp_mlp_train_step(tpp_mlp* net, const tpp_ctx* basis, const float* X,
                              const double* Mn, int32_t B, float lr, float* loss, void* stream);
/* device pointer to the gradients of the last train step (parameter layout) */
const float* tpp_mlp_gradients(const tpp_mlp* net);
/* Network inputs (X: device [E][2 n^2 + 1], may be NULL), normalised cores (Mn: device
 * [E][r*r] column-major, r = n + min(n^2 - n, n + 2), may be NULL) and block norms
 * ||A~||_F (norms: device [E]) of every element of a 2D context.  Asynchronous. */
tpp_status tpp_learned_inputs(const tpp_ctx* ctx, float* X, double* Mn, double* norms,
                              void* stream);
int32_t tpp_core_size(const tpp_ctx* ctx);                 /* r */
/* tpp_build_factors with the network's factors: every element whose predicted factors
 * have relative rank-2 error sqrt(L) <= threshold on its own block keeps them; the
 * others fall back to the exact KSVD.  Then the rest of the build as usual.  Needs a
 * 2D context with TPP_FEAT_LEARNED and a network of the same n.  report->num_fallback
 * counts the fallbacks.  Synchronises `stream`. */
tpp_status tpp_build_factors_learned(tpp_ctx* ctx, tpp_mlp* net, double threshold,
                                     tpp_build_report* report, void* stream);
/* Per-element loss L_e (device double [B]) of the network's factors for a batch
 * (X, Mn as for tpp_mlp_train_step); no gradients.  sqrt(L_e) is the relative
 * rank-2 error the learned build compares with its threshold.  Asynchronous. */
tpp_status tpp_mlp_element_loss(tpp_mlp* net, const tpp_ctx* basis, const float* X,
                                const double* Mn, int32_t B, double* loss, void* stream);
/* Learned preconditioner with both fallbacks: tpp_build_factors_learned(threshold),
 * then gmres_solve limited to iter_limit Arnoldi steps; if that solve has not
 * converged, the exact KSVD build (tpp_build_factors) and gmres_solve again from the
 * current x with the Arnoldi steps left of opts->max_iters (both solves together take
 * at most opts->max_iters).  result->iters counts both solves; *rebuilt = 1 when the
 * second build ran (report->num_fallback then equals num_elem).  Same argument rules
 * as the two calls. */
tpp_status tpp_solve_learned(tpp_ctx* ctx, tpp_mlp* net, double threshold, int32_t iter_limit,
                             const double* b, double* x, const tpp_gmres_opts* opts,
                             tpp_gmres_result* result, tpp_build_report* report,
                             int32_t* rebuilt, void* stream);

/* Number of DOFs and elements of the context's problem. */
int64_t tpp_num_dofs(const tpp_ctx* ctx);
int64_t tpp_num_elem(const tpp_ctx* ctx);

/* Arithmetic peak probe (instrumentation for rooflines): the rate in flop/s of 8
 * independent FMA chains per thread on 8 CTAs of 256 threads per SM, `iters` FMAs per
 * chain, prec TPP_FP64 (DFMA) or TPP_FP32 (FFMA), timed with CUDA events on `stream`
 * (synchronised).  The paper has no counterpart. */
tpp_status tpp_probe_fma_rate(int32_t prec, int32_t iters, double* flops, void* stream);

/* Number of CUDA kernels libtpp has launched since it was loaded (all contexts
 * and threads; instrumentation for benchmarks). */
int64_t tpp_kernel_launch_count(void);

/* Thread-local message of the last error (never NULL). */
const char* tpp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TPP_H */
