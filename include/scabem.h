/*
 * scabem: grid-accelerated PMCHW operator with a surface-conductive absorber,
 * for one NVIDIA GB300 (sm_103a).
 *
 * The operator is the boundary-element system of Zhang et al., "A Novel
 * Boundary Element Method Using Surface Conductive Absorbers for Full-Wave
 * Analysis of 3-D Nanophotonics": Galerkin-tested RWG currents on a closed
 * triangle mesh, PMCHW rows on plain surfaces (Eqs. 1-2), the modified rows
 * on the absorber surface (Eqs. 3, 13, 14) with the MPIE operators of
 * Eqs. 15-16.  Its matrix-vector product is evaluated by projecting the
 * currents onto a uniform grid, convolving with the interior and exterior
 * Helmholtz Green's functions by 3-D FFT, interpolating back, and adding a
 * near-field precorrection (the FFT acceleration of Appendix B, in the
 * precorrected-FFT form of the paper's reference Phillips97a).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Time dependence exp(+j w t) (Sec. II); outward normals.
 * - Lengths in micrometres.  Fields and currents are normalised so that the
 *   free-space impedance is 1: electric currents are eta0*J (V/m), magnetic
 *   currents M (V/m), tested H rows carry eta0*H.  Conductivities are passed
 *   in siemens and multiplied by eta0 = 376.730313668 ohm internally.
 * - Complex vectors are interleaved (re, im): complex64 (two floats) or
 *   complex128 (two doubles), column-major with leading dimension ld >= N.
 * - Unknown order (Appendix A): x = [J^L, M^L, J_e^R, J_i^R, M^R]; rows of
 *   A x = b: [Eq.1 (L edges), Eq.2 (L), Eq.3 (R), Eq.13 (R), Eq.14 (R)].
 *   Within a block, edges follow the canonical edge order: undirected edges
 *   sorted by (min vertex, max vertex); T+ of an edge is the triangle that
 *   traverses it from its smaller to its larger vertex.  An edge is an
 *   absorber ("R") edge iff both of its triangles carry region flag 1.
 * - Ownership: the caller owns every data buffer; the library owns handles
 *   and their device workspaces.  Handles are not thread-safe; work is
 *   ordered on the CUDA stream passed in (NULL = legacy default stream).
 * - Errors: every call returns a scabem_status; nothing aborts or throws
 *   across this interface.  scabem_last_error() describes the last failure
 *   of the calling thread.  There is no CPU fallback: without an sm_103
 *   device the calls return SCABEM_E_DEVICE.
 */
#ifndef SCABEM_H
#define SCABEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scabem_mesh* scabem_mesh_t;
typedef struct scabem_op* scabem_op_t;

typedef enum {
  SCABEM_OK = 0,
  SCABEM_E_ARG = -1,       /* invalid argument or size */
  SCABEM_E_MESH = -2,      /* open, non-manifold or degenerate mesh */
  SCABEM_E_DEVICE = -3,    /* no usable sm_103 device, or a CUDA error */
  SCABEM_E_NOMEM = -4,     /* device allocation failed */
  SCABEM_E_NOCONV = -5,    /* solver did not reach the tolerance */
  SCABEM_E_BREAKDOWN = -6, /* Krylov breakdown */
  SCABEM_E_NONFINITE = -7, /* NaN or Inf in an input or a residual */
  SCABEM_E_TIMEOUT = -8    /* a bounded device wait expired */
} scabem_status;

typedef enum { SCABEM_C64 = 0, SCABEM_C128 = 1 } scabem_prec;

/* Relative permittivity / permeability (real, positive) of the interior and
 * exterior media, and the free-space wavelength in um.  k_l = 2 pi
 * sqrt(eps_l mu_l)/lambda0, relative impedance z_l = sqrt(mu_l/eps_l). */
typedef struct {
  double eps_i, mu_i, eps_e, mu_e, lambda0;
} scabem_media;

/* Grid and discretisation options.
 *   n[3]      physical grid points per axis (x, y, z); the FFT size is 2n.
 *             Each 2n must be a power of two, in [8, 1024] along x and in
 *             [8, 512] along y and z.  The 2-D FFT planes (transverse = 1)
 *             need 2 n_y, 2 n_z <= 128 and (2 n_y)(2 n_z) <= 4096; larger
 *             planes always run as direct sums, which need the active
 *             columns' data (8 values each, plus the table of their offsets)
 *             to fit in one CTA's shared memory (SCABEM_E_ARG otherwise).
 *   h         grid spacing [um]; origin[3] coordinates of grid point 0.
 *   p         stencil points per axis (2, 3 or 4), Lagrange interpolation;
 *             every stencil must fall inside the physical grid.
 *   q         quadrature points per triangle (1, 3, 6 or 7; Dunavant rules).
 *   r_near    near-field radius [um]: triangle pairs with centroid distance
 *             below it get the exact panel interaction (precorrection).
 *   prec_mask bit 0: build complex64 operator data, bit 1: complex128.
 *   transverse how the (y, z) part of the grid convolution runs, per axis-0
 *             frequency: 1 = 2-D FFTs of the zero-padded planes with the
 *             Green spectrum; 2 = direct sum over the active (y, z) columns
 *             (those a stencil covers) with the axis-0 transform of the
 *             spatial Green table; 0 = automatic (direct when the active
 *             columns are few: nac^2 <= 16 (2 n_y)(2 n_z)).  Both give the
 *             same linear convolution up to rounding. */
typedef struct {
  int32_t n[3];
  double h;
  double origin[3];
  int32_t p;
  int32_t q;
  double r_near;
  int32_t prec_mask;
  int32_t transverse;
} scabem_grid_opts;

/* Create a mesh from host arrays: xyz (nv x 3, um), tri (nt x 3, vertex
 * indices, counter-clockwise seen from outside), region (nt; 0 = plain
 * surface with sigma = 0 (Sec. II "L"), 1 = absorber surface ("R")).
 * The mesh must be closed and consistently oriented (SCABEM_E_MESH).
 * Host-side topology only; no device memory is touched. */
int scabem_mesh_create(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt,
                       const int32_t* region, scabem_mesh_t* out);

/* Edge counts and the number of unknowns N = 2 n_L + 3 n_R. */
int scabem_mesh_info(scabem_mesh_t mesh, int64_t* n_edges_L, int64_t* n_edges_R, int64_t* n_unknowns);

/* Canonical edge table (host arrays of n_edges = n_L + n_R rows):
 * edge_v (ne x 2, min/max vertex), edge_t (ne x 2, T+ / T-), edge_class
 * (0 = L, 1 = R).  Any pointer may be NULL. */
int scabem_mesh_edges(scabem_mesh_t mesh, int64_t* edge_v, int64_t* edge_t, int32_t* edge_class);

void scabem_mesh_destroy(scabem_mesh_t mesh);

/* Build the operator on the current device: triangle geometry, quadrature,
 * stencils, the two Green's spectra (one 3-D FFT each) and the near-field
 * precorrection (closed-form panel integrals with singularity extraction,
 * minus the grid's own near interaction).  Conductivity starts at zero.
 * `stream` orders the set-up work; the call returns when it is complete. */
int scabem_op_create(scabem_mesh_t mesh, const scabem_media* media, const scabem_grid_opts* opts,
                     void* stream, scabem_op_t* out);

/* Sizes of the built operator: near pairs, bytes of near data per matvec in
 * the given precision, quadrature points. */
int scabem_op_info(scabem_op_t op, int64_t* n_near_pairs, int64_t* near_bytes_c64,
                   int64_t* near_bytes_c128, int64_t* n_qpoints);

/* Grid plan for scabem_op_create (host only; a convenience, not part of the
 * paper's method).  From the mesh's bounding box, picks per axis the smallest
 * power-of-two transform size 2n within the limits of scabem_grid_opts whose
 * physical grid holds the mesh and the stencil margin at a spacing no larger
 * than h_max [um] (e.g. the wavelength in the densest medium over 10), takes
 * the common spacing h = max over axes of extent / (n - p - 1.5) (so every
 * stencil stays inside, with 1.25 cells to spare on either side), centres the
 * mesh, and fills *opts: n, h, origin, p, q = 6, r_near = near_h * h (near_h
 * in grid steps, e.g. 2.05 or 3.05), prec_mask = 3, transverse = 0 (auto).
 * SCABEM_E_ARG for a null argument, h_max <= 0, p outside 2..4, near_h < 0,
 * or an h_max too small for the transform or (y, z) plane limits. */
int scabem_grid_plan(scabem_mesh_t mesh, double h_max, int32_t p, double near_h, scabem_grid_opts* opts);

/* Sparsity of the grid (Appendix B's uniform grid): physical grid points
 * that some projection stencil covers, and (i1, i2) columns holding one of
 * them.  Sources are zero and potentials unused elsewhere, so the axis-0
 * transforms run on the active columns only.  transverse_direct = 1 when the
 * (y, z) convolution runs as a direct sum over the active columns, 0 for 2-D
 * FFT planes.  Any output pointer may be NULL. */
int scabem_op_grid_info(scabem_op_t op, int64_t* n_covered_points, int64_t* n_active_columns,
                        int32_t* transverse_direct);

void scabem_op_destroy(scabem_op_t op);

/* Conductivity profile (Sec. IV, Eq. 23).
 *   SCABEM_SIGMA_MONOMIAL: sum over nseg segments of
 *       sigma0 * u(s)^d,  s = dir * (x_axis - x0) / L,  u = 0 for s < 0,
 *       u = s for 0 <= s <= 1, u = 1 for s > 1,
 *     seg[6*i .. 6*i+5] = {x0 [um], L [um], sigma0 [S], d, axis (0..2), dir (+1/-1)};
 *     d = 0 gives a step of height sigma0 at x0.
 *   SCABEM_SIGMA_PER_QPOINT: per_qpoint[t*q + a] [S], host array.
 *   SCABEM_SIGMA_BSPLINE: sum_k coef[k] N_k(s) [S], s = (x_axis - x0) / L,
 *     N_k the cubic B-splines on the clamped uniform knot vector of ncoef
 *     (>= 4, <= 1024) coefficients over [0, 1]; zero for s outside [0, 1].
 *     Uses x0 [um], L [um] (> 0), axis (0..2), ncoef and coef (host array,
 *     finite, >= 0).  A smooth profile for gradient studies with respect to
 *     the coefficients.
 * Conductivity enters only the Eq. 13 / Eq. 14 rows of absorber edges.
 * Fields a kind does not use are ignored. */
typedef enum {
  SCABEM_SIGMA_MONOMIAL = 0,
  SCABEM_SIGMA_PER_QPOINT = 1,
  SCABEM_SIGMA_BSPLINE = 2
} scabem_sigma_kind;
typedef struct {
  int32_t kind;
  int32_t nseg;
  const double* seg;
  const double* per_qpoint;
  double x0, L;
  int32_t axis, ncoef;
  const double* coef;
} scabem_sigma;
int scabem_set_sigma(scabem_op_t op, const scabem_sigma* sigma);

/* y = A x for nrhs right-hand sides.  x and y may be device or host memory
 * (host buffers are staged through device copies on `stream`).  prec selects
 * complex64 or complex128 arithmetic; the operator must have been built with
 * that precision.  Stream-ordered: returns after enqueueing (device buffers)
 * or after completion (host buffers).  The near-field stage waits on its
 * own bulk copies with a time limit (about a second); if one expires, that
 * launch's y is not valid and the next scabem_apply or scabem_solve on the
 * operator returns SCABEM_E_TIMEOUT (scabem_solve also reports it for its own
 * launches). */
int scabem_apply(scabem_op_t op, const void* x, void* y, int32_t nrhs, int64_t ld, int32_t prec, void* stream);

/* Circulant preconditioner for the plain-surface block of a straight guide
 * (Appendix B: A_LL of a mesh that repeats along the guide is block
 * Toeplitz over its regular slices; a block circulant approximation of it is
 * inverted with FFTs over the slice index, and the absorber rows keep the
 * block-diagonal preconditioner).  Slice k of the mesh spans
 * [x0 + k dx, x0 + (k + 1) dx) along `axis`; the plain-surface edges between
 * lateral (not end-cap) triangles of slices first .. first + count - 1 must
 * be translates of those of slice `first` (SCABEM_E_MESH otherwise).  Its
 * blocks come from the operator's own columns (complex128 operator when
 * built, else complex64): kind 0 takes Strang's circulant (the blocks of
 * offsets up to count / 2, wrapped; columns of the middle slice), kind 1
 * T. Chan's optimal circulant (each wrapped diagonal averaged, c_k =
 * ((R - k) T[k] + k T[k - R]) / R; columns of the first and last slice).  The
 * R = count DFT blocks (m x m, m = unknowns per slice) are inverted on the
 * device by Gauss-Jordan elimination with partial pivoting
 * (SCABEM_E_BREAKDOWN if one is singular).  From then on scabem_solve
 * (forward, transpose = 0) preconditions those unknowns with it; transposed
 * solves keep the block-diagonal preconditioner.  count = 0 removes it.
 * `mesh` must be the mesh the operator was built from; synchronises `stream`;
 * R m^2 complex128 values of device memory. */
typedef struct {
  int32_t axis;
  double x0, dx;
  int32_t first, count;
  int32_t kind; /* 0: Strang's circulant; 1: T. Chan's optimal circulant */
} scabem_circulant;
int scabem_set_precond_circulant(scabem_op_t op, scabem_mesh_t mesh, const scabem_circulant* c, void* stream);

/* The preconditioner that scabem_solve applies, z = M^-1 v (the inverse
 * per-edge diagonal blocks, and the circulant of scabem_set_precond_circulant
 * on its periodic unknowns unless transpose = 1), for nrhs complex128 device
 * columns of leading dimension ld; for tests and for callers that run their
 * own Krylov method.  Stream-ordered. */
int scabem_precond_apply(scabem_op_t op, const void* v, void* z, int32_t nrhs, int64_t ld, int32_t transpose,
                         void* stream);

/* Autotuner (a convenience, not part of the paper's method): times the
 * operator's runtime shape choices for an apply of nrhs (1..8) right-hand
 * sides in precision prec on the device, with CUDA events on `stream` (one
 * warm-up and five timed applies each, on an internal seeded vector), and
 * keeps the fastest for the operator's later applies and solves:
 *   - the (y, z) convolution: direct sums over the active columns or 2-D FFT
 *     planes, where both fit (the set-up builds both Green tables then);
 *   - the lines per CTA of the axis-0 transforms: 1, 2, 4, 8 or 16, as far
 *     as the transform length and shared memory allow.
 * out (host, 4 doubles): {best ms per apply, ms per apply of the
 * configuration found on entry, 1 if the direct sums won (0: FFT planes),
 * axis-0 lines per CTA}.  The results are the same linear operator in every
 * configuration (up to rounding).  Allocates and frees two vectors;
 * synchronises `stream`; on an error the operator keeps its configuration. */
int scabem_autotune(scabem_op_t op, int32_t prec, int32_t nrhs, void* stream, double* out);

/* Self-test of the bounded device waits behind SCABEM_E_TIMEOUT.  One warp
 * waits on an mbarrier that nothing ever completes, through the same wait
 * routine and limit (about a second) as the near-field record streams, and
 * reports the expiry through the operator's timeout flag as they do; the
 * call synchronises `stream` and then reads and clears that flag.  Expected
 * result: SCABEM_E_TIMEOUT, with the operator and the CUDA context still
 * usable.  SCABEM_OK would mean that the wait did not report its expiry
 * (a fault of the wait routine); SCABEM_E_ARG for a null operator;
 * SCABEM_E_TIMEOUT is also
 * returned (before launching) when an earlier launch had already expired. */
int scabem_selftest_wait_limit(scabem_op_t op, void* stream);

/* x = A^T y, the transpose (not the conjugate transpose) of the operator of
 * scabem_apply, for adjoint solves and gradients (reciprocity of the
 * Galerkin system).  The stages of scabem_apply run transposed in reverse
 * order: testing and row sums, near-field precorrection (over the source
 * triangles), interpolation (value and derivative stencils), the grid
 * convolution (each potential field with its medium's Green function),
 * projection and the current expansion.  Same arguments, layouts, host
 * staging and errors as scabem_apply, with y the input and x the output. */
int scabem_apply_adjoint(scabem_op_t op, const void* y, void* x, int32_t nrhs, int64_t ld, int32_t prec,
                         void* stream);

/* Excitation (Sec. II): kind 0 = plane wave (dir, pol), 1 = electric dipole
 * (pos, pol), 2 = complex-source-point beam at pos - j*b*dir radiating along
 * dir (pos, dir, b, pol).  side 0 = source in the interior medium (the
 * paper's case, Eqs. 8-9), 1 = exterior medium. */
typedef struct {
  int32_t kind;
  int32_t side;
  double pos[3];
  double dir[3];
  double pol[3];
  double b;
} scabem_source;

/* Tested right-hand side b (Appendix A) for nsrc sources into columns of b
 * (device or host, precision prec).  Uses the current conductivity. */
int scabem_rhs(scabem_op_t op, const scabem_source* src, int32_t nsrc, void* b, int64_t ld, int32_t prec,
               void* stream);

/* The same tested right-hand side as scabem_rhs, for callers that cannot
 * allocate device memory while they run (code inside another framework's
 * memory pool that has already reserved the device, real-time loops that
 * cannot take the device-wide synchronisation of a cudaFree, services that
 * must not hit out-of-memory mid-run).  The paper has no counterpart: this is
 * an interface variant, not part of the method.
 *   - b must be device memory (complex64 or complex128 per prec, ld >= N).
 *   - The per-call scratch (12 complex128 values per triangle) lives in one
 *     fixed device array of 32768 triangles (6 MiB), held by every GPU that
 *     loads the library until the process exits; meshes with more triangles
 *     are rejected with SCABEM_E_ARG.  No cudaMalloc, cudaFree or allocating
 *     library routine is called.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) once, with that device current; make that first
 *     call before any stream capture.
 *   - Every call shares the array: two calls whose work overlaps on the GPU
 *     (different streams, or different operators at once) race on it.  Each
 *     call writes every scratch entry it later reads, so the previous call's
 *     contents never leak into a result.
 *   - Work is enqueued on `stream`; the call does not synchronise. */
int scabem_rhs_noalloc(scabem_op_t op, const scabem_source* src, int32_t nsrc, void* b, int64_t ld, int32_t prec,
                       void* stream);

/* GMRES solve of A x = b (complex128 b and x, device or host; Appendix B's
 * iterative solver).  An outer loop forms the FP64 residual r = b - A x with
 * the complex128 operator and solves A d = r by restarted GMRES, x += d,
 * until |r|/|b| <= refine_tol or max_refine rounds.  prec = precision of the
 * operator inside GMRES: SCABEM_C128, or SCABEM_C64 (complex64 operator; needs
 * both precisions built).  The Krylov vectors are held as FP32 (hi, lo)
 * pairs, about 48 bits, with exact products and compensated sums; the
 * Hessenberg least squares, the norms and the refinement are FP64.  GMRES is right-preconditioned by the inverse per-edge diagonal
 * blocks of A (the block-diagonal preconditioner of Appendix B), rebuilt on
 * every scabem_set_sigma.  x holds the initial guess on entry; info reports
 * iterations, refinement rounds and the final FP64 relative residual.
 * transpose = 1 solves A^T x = b instead (the adjoint system of gradients),
 * with the transposed operator of scabem_apply_adjoint and the transposed
 * preconditioner blocks.  Returns SCABEM_E_NOCONV if refine_tol was not
 * reached. */
typedef struct {
  double tol;        /* relative residual of each inner GMRES solve */
  int32_t restart;   /* Krylov dimension, <= 200 */
  int32_t maxit;     /* total inner iterations */
  double refine_tol; /* outer FP64 relative residual */
  int32_t max_refine;
  int32_t prec;
  int32_t transpose; /* 0: A x = b, 1: A^T x = b */
} scabem_solve_opts;
typedef struct {
  int32_t iters;
  int32_t refinements;
  double relres;
  int32_t status;
} scabem_solve_info;
int scabem_solve(scabem_op_t op, const void* b, void* x, int32_t nrhs, int64_t ld, const scabem_solve_opts* opts,
                 void* stream, scabem_solve_info* info);

/* Gradient of lam^T (A x - b) with respect to the parameters of a
 * conductivity profile (A and b are affine in sigma: the sigma-weighted
 * terms of the Eq. 13 / Eq. 14 rows and of their incident-field right-hand
 * sides), summed over the quadrature points p:
 *   g_i = sum_p (d sigma_p / d c_i) d(lam^T (A x - b)) / d sigma_p.
 * x, lam: complex128, N each, device or host; src/nsrc: the excitation of b
 * (as for scabem_rhs; nsrc = 0 when b does not depend on sigma).  `basis`
 * names the parameters (only its shape is read):
 *   SCABEM_SIGMA_PER_QPOINT: Q entries, the per-point derivative itself [1/S];
 *   SCABEM_SIGMA_MONOMIAL:   nseg entries, d / d sigma0 of each segment;
 *   SCABEM_SIGMA_BSPLINE:    ncoef entries, d / d coef of each coefficient.
 * g_out: host, 2 * entries doubles (complex).  For x = A^-1 b and a real
 * objective J with dJ = Re(v^H dx), solve A^T lam = conj(v) (scabem_solve
 * with transpose = 1); then dJ/dc_i = -Re(g_i).  Needs the complex128
 * operator; synchronises `stream`. */
int scabem_sigma_gradient(scabem_op_t op, const void* x, const void* lam, const scabem_source* src, int32_t nsrc,
                          const scabem_sigma* basis, double* g_out, void* stream);

/* Interior electric field at npts host points (pts: npts x 3) from the
 * interior current set of x (complex128), plus the incident field of `inc`
 * if it is not NULL (Eq. 8: total interior field = E_inc + E_i(J_i, M_i)).
 * E_out: host, npts x 3 complex128 per right-hand side. */
int scabem_fields(scabem_op_t op, const void* x, int32_t nrhs, int64_t ld, const double* pts, int32_t npts,
                  const scabem_source* inc, double* E_out, void* stream);

/* Electric and magnetic field of one current set at npts host points
 * (pts: npts x 3), the operators of Eqs. 15-16 evaluated off the surface by
 * the triangle quadrature: side 0 = the interior set (J_i, -M) radiating in
 * the interior medium, plus the incident field of `inc` when it is not NULL
 * (Eq. 8: the total interior field); side 1 = the exterior set (J_e, M) in
 * the exterior medium (the total exterior field of an interior source; inc
 * is ignored).  x: complex128, device or host, nrhs columns of leading
 * dimension ld.  E_out, H_out: host, npts x 3 complex128 per right-hand
 * side, H in the eta0 = 1 scaling (eta0 H).  Needs the complex128 operator;
 * synchronises `stream`. */
int scabem_fields_eh(scabem_op_t op, const void* x, int32_t nrhs, int64_t ld, const double* pts, int32_t npts,
                     int32_t side, const scabem_source* inc, double* E_out, double* H_out, void* stream);

/* Decay rate by Poynting's theorem (Sec. III-B) at the cross-section
 * x = xc of a guide along x centred on y = z = 0:
 *   alpha = [ int_L' sigma |E_tan|^2 dl + Re oint_L (E x H*) . n dl ]
 *           / [ 2 Re int_A (E x H*) . x dS ],
 * A the rectangle |y| <= box[0], |z| <= box[1]; the core rectangle
 * |y| < core[0], |z| < core[1] takes the total interior field (with the
 * incident field of `inc` when not NULL), the rest of A and its outer
 * boundary L the exterior field.  Each of the nine rectangles uses n x n
 * Gauss-Legendre points, each side of L 2n.  The perimeter integral L' is
 * the surface integral of sigma eta0 |M|^2 over the band |x - xc| < slab of
 * the mesh, divided by its width 2 slab (|E_tan| = |n x M| = |M| on the
 * sheet), with the operator's own conductivity at each quadrature point.
 * x: complex128 (device or host); out (host, per right-hand side):
 * {alpha [1/um], loss per length, side flux per length, cross-section flux}.
 * Needs the complex128 operator; synchronises `stream`. */
typedef struct {
  double xc;
  double core[2];
  double box[2];
  double slab;
  int32_t n;
} scabem_poynting;
int scabem_poynting_rate(scabem_op_t op, const void* x, int32_t nrhs, int64_t ld, const scabem_poynting* p,
                         const scabem_source* inc, double* out, void* stream);

/* Reflection on a line of probe points inside the guide (Sec. I, Table 1):
 * samples the component `comp` of the total interior field at npts points
 * p0 + t * e_axis, t in [t0, t1]; fits E = a exp(-j beta t) + c exp(j beta t)
 * by least squares (beta scanned over nbeta values in [beta_lo, beta_hi], or
 * fixed when nbeta == 1) and reports r = c/a.  Also returns the standing-wave
 * ratio max|E|/min|E| and (SWR-1)/(SWR+1).
 * out (host, per rhs): {Re r, Im r, beta, residual, SWR, r_swr}. */
typedef struct {
  int32_t axis;
  int32_t comp;
  double p0[3];
  double t0, t1;
  int32_t npts;
  double beta_lo, beta_hi;
  int32_t nbeta;
} scabem_probe;
int scabem_reflection(scabem_op_t op, const void* x, int32_t nrhs, int64_t ld, const scabem_probe* probe,
                      const scabem_source* inc, double* out, void* stream);

/* Decay-rate fit (Sec. III: the field inside a guide with uniform surface
 * conductivity decays along the axis).  Least squares for
 *   E(t) = a exp(-g tau) + c exp(g tau),  g = alpha + j beta,
 *   tau = t - (t_first + t_last) / 2,
 * both waves decaying along their direction of travel, over the uniform grid
 * of nalpha x nbeta candidates (alpha in [alpha_lo, alpha_hi] [1/um], beta in
 * [beta_lo, beta_hi] [rad/um], end points included; the low value alone when
 * the count is 1).  For each candidate the amplitudes solve the 2 x 2 normal
 * equations; the candidate with the smallest residual wins (ties: the first
 * in alpha-major order).
 *   scabem_decay_fit: given samples, host arrays t (npts, [um]) and E (npts
 *   complex128, interleaved); npts >= 4, nalpha * nbeta <= 2^24;
 *   SCABEM_E_NONFINITE for a non-finite sample, SCABEM_E_DEVICE without a
 *   GB300.
 *   scabem_decay_rate: the samples are the total interior field component
 *   `comp` on the probe line of scabem_reflection (its beta range is used),
 *   for each right-hand side; needs the complex128 operator.
 * out (host, 6 per fit): {alpha, beta, relative residual, Re(c/a), Im(c/a),
 * |a|}, with a and c referred to the midpoint of the samples. */
int scabem_decay_fit(const double* t, const double* E, int32_t npts, double alpha_lo, double alpha_hi,
                     int32_t nalpha, double beta_lo, double beta_hi, int32_t nbeta, double* out, void* stream);
int scabem_decay_rate(scabem_op_t op, const void* x, int32_t nrhs, int64_t ld, const scabem_probe* probe,
                      double alpha_lo, double alpha_hi, int32_t nalpha, const scabem_source* inc, double* out,
                      void* stream);

/* Stage timing of scabem_apply (instrumentation, not part of the paper's
 * method).  While enabled, every apply records CUDA events at its stage
 * boundaries on its own stream, for at most max_applies applies (events are
 * created here, so enable before any stream capture).  scabem_profile_read
 * waits for the recorded events, returns per-stage summed milliseconds in
 * stage_ms[6] = {summaries and point sources, projection, FFT axis-0
 * forward, (y, z) convolution with the Green functions (direct sums or FFT
 * planes), FFT axis-0 inverse, points (interpolation + near field + testing
 * + row sums)} and the number of applies, and starts a new record.
 * enable = 0 releases the events. */
int scabem_profile(scabem_op_t op, int32_t enable, int32_t max_applies);
int scabem_profile_read(scabem_op_t op, double* stage_ms, int64_t* n_applies);

/* Arithmetic peak of the current GPU's fused multiply-add pipe (instrumentation,
 * not part of the paper's method): a kernel of independent FMA chains in
 * registers, with no memory traffic, 8 CTAs of 256 threads per SM, timed with
 * CUDA events on `stream` (the second of two launches).  prec = SCABEM_C128:
 * FP64 FMA (the pipe of the complex128 operator); SCABEM_C64: packed FP32x2
 * FMA (the pipe of the complex64 operator).  *tflops: measured TFLOP/s.
 * Allocates and frees a small device buffer; synchronises `stream`. */
int scabem_peak_fma(int32_t prec, double* tflops, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* scabem_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SCABEM_H */
