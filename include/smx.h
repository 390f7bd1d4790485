/*
 * smx.h -- C ABI of the GB300 (sm_103a) leapfrog for the spline geometric
 * discretisation of Maxwell's equations of Kapidani & Vazquez, "High order
 * geometric methods with splines: fast solution with explicit time-stepping
 * for Maxwell equations" (arXiv 2302.04979), scheme 2 (Sec. 3.4).
 *
 * Conventions shared by every call
 * --------------------------------
 * Fields (Sec. 2.4, field placement; Sec. 3.1):
 *   E in X^1_{h,0} (primal 1-forms, degrees p-1/p, zero tangential trace)
 *   B in X^2_{h,0} (primal 2-forms)
 *   H in X~^1      (dual 1-forms, degrees p-2/p-1)
 *   D in X~^2      (dual 2-forms)
 * len(e) = len(d) = N_e and len(b) = len(h) = N_h (dim X^1_{h,0} = dim X~^2,
 * dim X^2_{h,0} = dim X~^1, Sec. 2.3).  With n_a = nel_a + p_a:
 *   E/D component c has (n-1) functions along axis c and (n-2) along the others;
 *   B/H component c has (n-2) functions along axis c and (n-1) along the others.
 * Layout: the three components are stored one after the other (x, y, z; for
 * 2-forms the coefficients of dy^dz, dz^dx, dx^dy); inside a component the
 * index is i + N_x (j + N_y k) -- x fastest, the vec convention of Sec. 4.2.
 * All field pointers are DEVICE pointers to FP64 arrays owned by the caller
 * (normally torch tensors); the library never allocates device memory.
 * All device work is enqueued on the stream set with smx_set_stream (default
 * the legacy default stream) and returns after enqueue unless stated.
 * Every call returns SMX_OK (0) or a negative status; smx_strerror names it.
 * A call that fails argument checks enqueues nothing.  Unless a call lists
 * its own errors, these are the only ones it returns: SMX_EINVAL (a null
 * context or pointer, an out-of-range field, axis, class or count),
 * SMX_ESTATE (the call needs a bound workspace and none is bound), SMX_ECUDA
 * (a launch, copy or event call failed).
 */
#ifndef SMX_H
#define SMX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SMX_OK 0
#define SMX_EINVAL (-1)      /* bad argument: p < 2, nel < 1, null pointer, nsteps < 0, dt <= 0 ... */
#define SMX_EGEOM (-2)       /* det J_F <= 0 (or non-finite) at some quadrature point */
#define SMX_EMAT (-3)        /* eps or mu <= 0 or non-finite */
#define SMX_ECUDA (-4)       /* a CUDA runtime call failed (launch, copy, ...) */
#define SMX_ENONFINITE (-5)  /* a reduction saw NaN or Inf in the fields */
#define SMX_ESTATE (-6)      /* workspace missing or too small */
#define SMX_ENOMEM (-7)      /* host allocation failed */
#define SMX_ESINGULAR (-8)   /* a 1D pairing factor has a (near) zero pivot */
#define SMX_ENOSPACE (-9)    /* problem larger than the library's fixed device array (SMX_NOALLOC_BYTES) */
#define SMX_ETIMEOUT (-10)   /* a device-side wait gave up after its time limit (see smx_device_status) */

/* ---- geometry map F : (0,1)^3 -> Omega (Sec. 2.3) ---- */
#define SMX_GEOM_IDENTITY 0  /* F = identity: the unit-cube cavity of Sec. 5.1.1 */
#define SMX_GEOM_SINE_BUMP 1 /* F_i = x_i + a sin(pi x) sin(pi y) sin(pi z), a = geom_amplitude */
#define SMX_GEOM_CALLBACK 2  /* a general single-patch map given by the host callback geom_fn (Sec. 2.3) */

/* Host callback of SMX_GEOM_CALLBACK: for i < n, the map F at the parametric
 * point (xhat[3i], xhat[3i+1], xhat[3i+2]) in (0,1)^3 into x[3i + r] = F_r and
 * its Jacobian into jac[9i + 3r + c] = dF_r / dxhat_c.  Called inside
 * smx_create (at every quadrature point, a few calls of many points) and
 * smx_project; det J_F must be positive and every value finite there
 * (SMX_EGEOM otherwise).  A map that is not the identity always takes the
 * quadrature Hodge (sum-factorised, metric w J^T J / det J stored per point). */
typedef void (*smx_geometry_fn)(int64_t n, const double* xhat, double* x, double* jac, void* user);

/* ---- material description (eps or mu) ---- */
#define SMX_MAT_CONST 0      /* one value everywhere */
#define SMX_MAT_BLOCKS 1     /* piecewise constant on a grid of element blocks aligned with the mesh */
#define SMX_MAT_POINTWISE 2  /* host callback evaluated at the physical quadrature points (setup only) */

/* ---- field selectors ---- */
#define SMX_FIELD_E 0
#define SMX_FIELD_B 1
#define SMX_FIELD_H 2
#define SMX_FIELD_D 3

/* Host callback for SMX_MAT_POINTWISE: out[i] = material at the physical point
 * (xyz[3i], xyz[3i+1], xyz[3i+2]), i < n.  Called only inside smx_create. */
typedef void (*smx_material_fn)(int64_t n, const double* xyz, double* out, void* user);

typedef struct {
    int kind;                   /* SMX_MAT_* */
    double value;               /* SMX_MAT_CONST */
    int blocks[3];              /* SMX_MAT_BLOCKS: block counts along x, y, z; each divides nel */
    const double* block_values; /* SMX_MAT_BLOCKS: host array, blocks[0]*blocks[1]*blocks[2], x fastest */
    smx_material_fn fn;         /* SMX_MAT_POINTWISE */
    void* user;                 /* passed to fn */
} smx_material;

typedef struct {
    int p[3];              /* spline degree per axis, p >= 2 (Sec. 2.3; per-axis degrees, Eq. tensor_K) */
    int nel[3];            /* uniform elements per axis, nel >= 1 (maximal smoothness, Sec. 5) */
    int geometry;          /* SMX_GEOM_* */
    double geom_amplitude; /* SMX_GEOM_SINE_BUMP amplitude a; |a| < 1/(3 pi) keeps det J_F > 0 */
    smx_material eps;      /* permittivity: weights M~^2_{1/eps} (Eq. discrete2_hodge_eps) */
    smx_material mu;       /* permeability: weights M^2_{1/mu} (Eq. discrete2_hodge_mu) */
    int precision;         /* SMX_FP64, SMX_MIXED or SMX_MIXED_REFINED: arithmetic of smx_step / smx_step_host */
    smx_geometry_fn geom_fn; /* SMX_GEOM_CALLBACK: the map (must stay callable while smx_project may be called) */
    void* geom_user;         /* passed to geom_fn */
    int scheme1;           /* nonzero: also build the tables of scheme 1 (smx_step_scheme1; p <= 5) */
} smx_params;

/* ---- precision of the leapfrog step ----
 * SMX_FP64: every operation in FP64.
 * SMX_MIXED: the stepped state d, b and its updates stay FP64 (one FP64 FMA
 * per coefficient per half step); the curl differences, the Hodge mass apply
 * and the pairing sweeps run in FP32 with operator coefficients stored as
 * FP32 (hi, lo) pairs (hi + lo = the FP64 value to about 2^-48), so only the
 * data is rounded to FP32.  On a curved map or with pointwise material the
 * quadrature metric is stored in FP32 (rounded once).  Only smx_step /
 * smx_step_host (and smx_hodge_star_mixed) change; every other call stays FP64. */
#define SMX_FP64 0
#define SMX_MIXED 1
/* SMX_MIXED_REFINED: the mixed operators with one refinement sweep of each
 * Kronecker solve whose residual is formed in FP64.  Every Hodge star runs
 * y = M x (FP32 element contributions summed in FP64), x0 = K^{-1} y in FP32,
 * r = y - K x0 in FP64 (banded 1D pairing factors on the FP64 pipe),
 * c = K^{-1} r in FP32 and writes x0 + c in FP64; the state d, b, e, h and
 * the curls are FP64.  The line operators are those of SMX_MIXED (CUDA-core
 * or tensor-core dense A^{-1} products, selected by smx_set_mode_kernel). */
#define SMX_MIXED_REFINED 2

typedef struct smx_ctx smx_ctx;

/* Build a context: knots, 1D pairing matrices G-hat, M-hat and their banded LU
 * (Sec. 4.1-4.3, Table 1 setup rows), Hodge tables (1D masses or quadrature
 * metric) -- all on the host in FP64.  Owns host memory only.
 * Errors: SMX_EINVAL, SMX_EGEOM, SMX_EMAT, SMX_ESINGULAR, SMX_ENOMEM. */
int smx_create(const smx_params* params, smx_ctx** out);

/* Free the context's host memory (the bound workspace stays the caller's). */
int smx_destroy(smx_ctx* ctx);

/* Static text for a status code. */
const char* smx_strerror(int status);

/* N_e = dim X^1_{h,0} = dim X~^2, N_h = dim X^2_{h,0} = dim X~^1 (Sec. 2.3). */
int smx_sizes(const smx_ctx* ctx, int64_t* n_e, int64_t* n_h);

/* Shape of component comp of a field: shape[0] = N_x, shape[1] = N_y, shape[2] = N_z. */
int smx_comp_shape(const smx_ctx* ctx, int field, int comp, int64_t shape[3]);

/* Device workspace size in bytes (tables + scratch).  The caller allocates it
 * (256-byte aligned) and binds it; the library never calls cudaMalloc. */
int smx_workspace_bytes(const smx_ctx* ctx, size_t* bytes);

/* Bind device memory of at least smx_workspace_bytes bytes and upload the
 * tables into it (synchronous on the context stream).  Errors: SMX_ESTATE if
 * too small or misaligned, SMX_ECUDA. */
int smx_bind_workspace(smx_ctx* ctx, void* device_ptr, size_t bytes);

/* Stream for all later device work (a cudaStream_t passed as void*; NULL =
 * legacy default stream). */
int smx_set_stream(smx_ctx* ctx, void* stream);

/* ==== Scheme 1 (Sec. 3.3): Hodge stars by mass-matrix solves ====
 * The comparison scheme of the paper: the same kick-drift-kick leapfrog on (d, b), with
 *   e = (M^1_eps)^{-1} K~_2 d  (Eq. discrete1_hodge_eps),  h = (M~^1_mu)^{-1} K_2 b  (Eq. discrete1_hodge_mu),
 * M^1_eps the mass of X^1_{h,0} weighted by eps (1-form pullback u = J^{-T} u^, Sec. 2.3), M~^1_mu
 * that of X~^1 weighted by mu, K~_2 = K_1^T and K_2 = K~_1^T (Eq. pairing_transpose).  Each mass
 * solve is a conjugate-gradient iteration on the device (matrix-free mass apply: block-Kronecker
 * on the identity map, sum-factorised quadrature otherwise) preconditioned with the unit-material
 * Kronecker mass (three banded line sweeps; exact up to the material constant on the identity map
 * with constant material), stopped at ||y - M x|| <= tol ||y||; the host reads the residual every
 * four iterations, so these calls synchronise the stream.  The context must be created with
 * scheme1 = 1 (else SMX_ESTATE).  Vectors as for smx_step; e and h are written. */

/* One scheme-1 Hodge star: field SMX_FIELD_D gives out = e from x = d, SMX_FIELD_B gives out = h
 * from x = b.  *iters (optional): CG iterations used.  Errors: SMX_EINVAL, SMX_ESTATE,
 * SMX_ESINGULAR (no convergence in maxit iterations), SMX_ENONFINITE, SMX_ECUDA. */
int smx_scheme1_star(smx_ctx* ctx, int field, const double* x, double* out, double tol, int maxit, int* iters);

/* nsteps kick-drift-kick steps of scheme 1 (the order of smx_step); *max_iters (optional): the
 * largest CG iteration count of any solve.  Errors as smx_scheme1_star and smx_step. */
int smx_step_scheme1(smx_ctx* ctx, double* d, double* b, double* e, double* h, const double* jhat,
                     const double* amp, double dt, int nsteps, double tol, int maxit, int* max_iters);

/* E_h = 1/2 (e^T K~_2 d + h^T K_2 b) of scheme 1 (Sec. 3.3; equal to 1/2 (e^T M^1 e + h^T M~^1 h)
 * when e, h are the stars of d, b).  Synchronises.  out[0] receives it.
 * Errors: SMX_EINVAL, SMX_ESTATE (no workspace, or not a scheme-1 context), SMX_ENONFINITE,
 * SMX_ECUDA. */
int smx_energy_scheme1(smx_ctx* ctx, const double* d, const double* b, const double* e, const double* h,
                       double* out);

/* CFL limit of scheme 1 (Sec. 5.2): 2 / sqrt(lambda_max) of D~^1 S_H D^1 S_E by power iteration (as
 * smx_cfl; v, w of N_e, t of N_h, device), with the mass solves to cg_tol in at most cg_maxit
 * iterations.  Errors: those of smx_scheme1_star (a mass solve), SMX_ENONFINITE (a non-finite or
 * non-positive Rayleigh quotient). */
int smx_cfl_scheme1(smx_ctx* ctx, int iters, double tol, double* v, double* w, double* t, double cg_tol,
                    int cg_maxit, double* dt_max);

/* CUDA graphs for smx_step (default on): the first call with a given set of
 * (d, b, e, h, jhat, amp) pointers, dt and nsteps is captured into a graph,
 * later identical calls replay it with one launch.  Only the last call is
 * cached; a different argument set recaptures.  Eager launches are used when
 * per-kernel timing is on or the stream is the legacy default stream (NULL),
 * which cannot be captured.  enable = 0 always launches eagerly. */
int smx_set_graphs(smx_ctx* ctx, int enable);

/* Kernel for the line operators of the Hodge stars (Eq. kroninverse per axis).
 * Mixed steps (SMX_MIXED, SMX_MIXED_REFINED, every line length <= 80; dense products):
 *   SMX_MODE_TENSOR: tcgen05 tensor cores by exact digit slicing with four
 *     digits -- lines and operator rows as 31-bit fixed-point integers, the
 *     four digit levels accumulated exactly, one rounding to FP32 at the end
 *     (more accurate than an FP32 dot product, no accumulation bias);
 *   SMX_MODE_SIMT: FP32 CUDA cores with the operator as FP32 (hi, lo) pairs;
 *   SMX_MODE_AUTO (default): the tensor cores once lines reach 32 entries,
 *     else the CUDA cores (faster for short lines).
 * FP64 step (SMX_FP64):
 *   SMX_MODE_TENSOR (every line length <= 80): the dense operator applied on
 *     the tcgen05 tensor cores by exact digit slicing -- lines and operator
 *     rows as 55-bit fixed-point integers in seven balanced base-256 BF16
 *     digits, each digit level accumulated exactly in FP32 -- with the
 *     rounding error bound of an FP64 dot product;
 *   SMX_MODE_SIMT: banded LU recurrences on the FP64 pipe (any line length);
 *   SMX_MODE_AUTO (default): per star, the faster of the two as measured on
 *     GB300 -- the tensor-core products once lines reach 48 entries, for a
 *     separable star (fused mass + solve) and, from degree 4 or from lines of
 *     64 entries, for the pairing sweeps after a mass apply; the banded
 *     recurrences otherwise.
 * The selection applies where the context has dense operators; elsewhere the
 * banded recurrences run.  Errors: SMX_EINVAL. */
#define SMX_MODE_TENSOR 0
#define SMX_MODE_SIMT 1
#define SMX_MODE_AUTO 2
int smx_set_mode_kernel(smx_ctx* ctx, int which);
/* The line-operator selection in effect: the setting above where the
 * context has dense operators (every line length <= 80; SMX_MODE_AUTO of a
 * mixed context reads the kernel it selects), else SMX_MODE_SIMT.  Host only.
 * Errors: SMX_EINVAL. */
int smx_mode_kernel(const smx_ctx* ctx, int* which);

/* Synchronise the context stream and read the device status word: SMX_OK, or
 * SMX_ETIMEOUT if a kernel of this context gave up a bounded device-side wait
 * (the tensor-core completion wait, one second) since the last call; the word
 * is then cleared.  Results of the affected launches are not valid. */
int smx_device_status(smx_ctx* ctx);

/* b += alpha * D^1 e: primal curl by the +-1 incidence matrix (Eq. discrete2_faraday,
 * Remark on incidence matrices after Table 1).  e: N_e, b: N_h, device, no aliasing.
 * Errors: SMX_EINVAL, SMX_ESTATE, SMX_ECUDA (likewise the four calls below). */
int smx_curl_primal(smx_ctx* ctx, const double* e, double* b, double alpha);

/* d += alpha * (D~^1 h - s * jhat): dual curl plus the current source
 * (Eq. discrete2_ampere).  jhat (N_e, device) may be NULL, then s is ignored. */
int smx_curl_dual(smx_ctx* ctx, const double* h, double* d, double alpha,
                  const double* jhat, double s);

/* y = M x, the Hodge mass apply: field SMX_FIELD_B -> M^2_{1/mu} (N_h),
 * SMX_FIELD_D -> M~^2_{1/eps} (N_e) (Eq. discrete2_hodge_mu / _eps right-hand
 * sides, Sec. 3.4).  Matrix free; y is overwritten; x and y must not alias. */
int smx_hodge_apply(smx_ctx* ctx, int field, const double* x, double* y);

/* x = K^{-1} y, the pairing solve by per-axis 1D banded solves (Sec. 4.2,
 * Eq. kroninverse): which = SMX_FIELD_E solves K_1 e = y (y in the D layout,
 * N_e); which = SMX_FIELD_H solves K~_1 h = y (y in the B layout, N_h).
 * y is left unchanged; x may equal y (in place). */
int smx_pairing_solve(smx_ctx* ctx, int which, const double* y, double* x);

/* One discrete Hodge star of scheme 2: e = K_1^{-1} M~^2_{1/eps} d (field SMX_FIELD_D,
 * out = e) or h = K~_1^{-1} M^2_{1/mu} b (field SMX_FIELD_B, out = h)
 * (Eq. discrete2_hodge_eps / _mu).  Uses the workspace scratch. */
int smx_hodge_star(smx_ctx* ctx, int field, const double* x, double* out);

/* nsteps kick-drift-kick leapfrog steps of scheme 2 (Sec. 3.4, Sec. 4.2):
 *   b -= dt/2 D^1 e;  h = K~_1^{-1} M b;  d += dt (D~^1 h - amp[n] jhat);
 *   e = K_1^{-1} M~ d;  b -= dt/2 D^1 e.
 * d, e: N_e; b, h: N_h; device, updated in place.  On entry e must be
 * consistent with d (e.g. from smx_hodge_star); on return e is consistent
 * with the new d and h holds the last half-step value.  jhat (N_e) and amp
 * (nsteps values, amp[n] = s(t_n + dt/2)) are device arrays; jhat = NULL
 * means J = 0 (amp ignored).  Errors: SMX_EINVAL (dt <= 0 or non-finite,
 * nsteps < 0), SMX_ESTATE, SMX_ECUDA. */
int smx_step(smx_ctx* ctx, double* d, double* b, double* e, double* h,
             const double* jhat, const double* amp, double dt, int nsteps);

/* Energies at a synchronised time (Eq. energy_matrix_wedge, Sec. 3.4):
 * out[0] = E_h = 1/2 (d^T M~ d + b^T M b);
 * out[1] = W = E_h - dt^2/8 (D^1 e)^T M (D^1 e), the quantity the leapfrog
 * conserves exactly (e may be NULL: then out[1] = out[0]).
 * Synchronises the stream.  Returns SMX_ENONFINITE if a sum is NaN or Inf. */
int smx_energy(smx_ctx* ctx, const double* d, const double* b, const double* e,
               double dt, double out[2]);

/* Largest stable leapfrog dt: 2/sqrt(lambda_max) of L M L^T M~ with
 * L = D~^1 K~_1^{-1} (Sec. 5.2 CFL), by power iteration on the device from a
 * fixed pseudo-random start; stops after iters or when the Rayleigh quotient
 * changes by less than tol (relative).  Uses 3 device vectors of the caller:
 * v (N_e), w (N_e), t (N_h).  Synchronises the stream.
 * Errors: SMX_EINVAL, SMX_ESTATE, SMX_ENONFINITE (a non-finite or non-positive
 * Rayleigh quotient), SMX_ECUDA. */
int smx_cfl(smx_ctx* ctx, int iters, double tol, double* v, double* w, double* t,
            double* dt_max);

/* nsteps leapfrog steps on HOST state: copies d, b, e (host, FP64) into the
 * workspace's state vectors, runs smx_step there, copies d, b, e, h back and
 * synchronises.  Host buffers should be pinned for asynchronous copies.
 * jhat and amp as in smx_step (device pointers or NULL).  On an error the
 * stream is synchronised before the return, so no copy is left reading or
 * writing the host buffers; an error of the step itself leaves d, b, e, h
 * unchanged.  Errors: those of smx_step, SMX_ECUDA (a copy). */
int smx_step_host(smx_ctx* ctx, double* d, double* b, double* e, double* h,
                  const double* jhat, const double* amp, double dt, int nsteps);

/* Host callback for smx_project: out[3i + c] = component c of the physical
 * vector proxy of a 2-form at the physical point (xyz[3i], xyz[3i+1],
 * xyz[3i+2]), i < n. */
typedef void (*smx_field_fn)(int64_t n, const double* xyz, double* out, void* user);

/* L2 projection of a physical 2-form (initial data and the source profile by
 * projection, Sec. 5.1.1) onto X~^2 (field = SMX_FIELD_D, coefficients d or
 * jhat; N_e values) or X^2_{h,0} (SMX_FIELD_B, coefficients b; N_h values).
 * Through the Piola map of 2-forms the right-hand side is
 * r_i = int (J^T V) . vhat_i dxhat and the coefficients solve M_1 x = r with
 * the unweighted 2-form mass (Sec. 3.4 with gamma = 1); Gauss-Legendre with
 * p + 1 points per element and axis.  Solved on the host in FP64 by conjugate
 * gradients preconditioned with the identity-map mass (exact on the identity
 * map), to a relative residual of 1e-14.  fn is called once per slab of
 * elements along z.  Host only: no workspace or GPU needed; coeffs is a host
 * array.  Errors: SMX_EINVAL (field, null pointers), SMX_ENONFINITE (fn
 * returned a non-finite value), SMX_ESINGULAR (no convergence in 500
 * iterations). */
int smx_project(const smx_ctx* ctx, int field, smx_field_fn fn, void* user, double* coeffs);

/* Kernel accounting for benchmarks.  smx_launch_count returns the number of
 * device kernels this context has launched so far (memsets and copies are not
 * counted).  smx_set_timing(ctx, 1) brackets every later launch with CUDA
 * events on the context stream; smx_kernel_times synchronises, adds up the
 * bracketed durations per kernel class and clears them:
 *   0 curl_primal, 1 curl_dual, 2 hodge_block, 3 hodge_quad,
 *   4 solve along x, 5 solve along y, 6 solve along z, 7 reductions,
 *   8/9/10 fused mass + solve along x/y/z (separable Hodge star),
 *   11 curl_primal and 12 curl_dual of the mixed step (FP32 differences),
 *   13 FP32 block Hodge, 14/15/16 FP32 line passes along x/y/z, 17 casts,
 *   18 FP32 quadrature Hodge, 19 per-block mass derivative (reverse step),
 *   20 receivers and small vector updates,
 *   21/22/23 FP64 dense line operators on the tensor cores along x/y/z,
 *   24/25/26 the mixed step's dense line operators on the tensor cores along x/y/z,
 *   27 the refined step's FP64 residual passes.
 * ms[SMX_NCLASS] receives milliseconds, counts[SMX_NCLASS] launches per class. */
#define SMX_NCLASS 28
int smx_launch_count(const smx_ctx* ctx, int64_t* n);
int smx_set_timing(smx_ctx* ctx, int enable);
int smx_kernel_times(smx_ctx* ctx, double* ms, int64_t* counts);

/* Algorithmic work of ONE launch of kernel class cls (numbering above) on
 * field (SMX_FIELD_*: the field the launch writes -- B or H for curl_primal /
 * solves of K~_1 / the M^2 Hodge, D or E for curl_dual / solves of K_1 / the
 * M~^2 Hodge): FP64 flops the kernel's algorithm performs (an FMA counts 2)
 * and the bytes it must move to and from device memory at minimum (each input
 * read once, each output written once).  SMX_EINVAL for a class that the
 * context does not launch for that field. */
int smx_kernel_work(const smx_ctx* ctx, int cls, int field, double* flops, double* bytes);

/* Allocation-free variant of smx_hodge_star, for callers that cannot allocate
 * device memory at all -- code running where cudaMalloc is unavailable or
 * forbidden (inside another library's memory pool, a sandboxed plug-in, a
 * process whose allocator is owned by someone else) and that therefore cannot
 * provide the workspace the other calls need.  The paper has no counterpart;
 * this is a deployment convenience.
 *
 * Computes the same result as smx_hodge_star (e = K_1^{-1} M~ d for
 * SMX_FIELD_D, h = K~_1^{-1} M b for SMX_FIELD_B) with the caller passing only
 * the input x and the output out (device, FP64).  The tables and the
 * intermediate vector live in one fixed array of SMX_NOALLOC_BYTES (16 MiB)
 * that the library image reserves on every GPU that loads it, until the
 * process exits.  No workspace needs to be bound, and the call itself makes
 * no device allocation (no cudaMalloc, cudaFree or allocating library call).
 *
 * Limits and behaviour:
 *  - the context's tables plus one field vector must fit in SMX_NOALLOC_BYTES,
 *    otherwise SMX_ENOSPACE (about 0.9M degrees of freedom per field at p = 3);
 *  - only the block-Kronecker Hodge (identity map, constant or block material)
 *    is supported: the quadrature tables of curved maps or pointwise
 *    materials are too large, and the call returns SMX_EINVAL;
 *  - the first call on a device looks up the array's device address (with that
 *    device current); make that first call before any stream capture;
 *  - the array used is the current device's: the context stream (if not the
 *    legacy default stream) must belong to the current device, else SMX_EINVAL;
 *  - a material update (smx_set_material_blocks) takes effect here too: the
 *    next call re-uploads the context's tables;
 *  - the array is shared by every context and every call on the device and
 *    keeps the last call's contents; a call re-uploads its context's tables
 *    (an asynchronous host-to-device copy on the context stream) when another
 *    context used the array last, and clears the intermediate vector itself;
 *  - calls that overlap on the GPU (different streams, or different contexts
 *    without ordering between them) race on the array; serialise them.
 * Errors: SMX_EINVAL (null argument, field not B or D, quadrature Hodge,
 * stream of another device), SMX_ENOSPACE, SMX_ECUDA. */
#define SMX_NOALLOC_BYTES (16u << 20)
int smx_hodge_star_noalloc(smx_ctx* ctx, int field, const double* x, double* out);

/* Diagnostics for tests: copy the host-side banded LU of one 1D factor.
 * axis 0..2; which 0 = G-hat, 1 = M-hat, 2 = G-hat^T, 3 = M-hat^T (Sec. 4.1).
 * dense_out receives the n x n factor matrix A (row-major) rebuilt from the
 * stored L and U, so tests can compare it with the definition. */
int smx_factor_matrix(const smx_ctx* ctx, int axis, int which, int64_t* n, double* dense_out);

/* Which Hodge kernels a field uses: 0 = block-Kronecker mass apply (identity
 * map, block-constant material) followed by the pairing sweeps; 1 = quadrature
 * mass apply (curved map or pointwise material) followed by the sweeps; 2 =
 * constant material on the identity map: the mass is one Kronecker product and
 * the Hodge star runs as three fused mass + solve line passes (the plain mass
 * apply still uses the block kernel). */
int smx_hodge_mode(const smx_ctx* ctx, int field, int* mode);

/* The Hodge star of the mixed step on its own (Eq. discrete2_hodge_eps /
 * discrete2_hodge_mu in mixed precision): out = K_1^{-1} M~ x (SMX_FIELD_D) or
 * K~_1^{-1} M x (SMX_FIELD_B) computed by the FP32 kernels smx_step uses for
 * SMX_MIXED (x read as FP64, result FP32 widened into the FP64 out; device
 * arrays).  Errors: SMX_EINVAL, SMX_ESTATE (no workspace, or the context is
 * not SMX_MIXED), SMX_ECUDA. */
int smx_hodge_star_mixed(smx_ctx* ctx, int field, const double* x, double* out);

/* ==== Reverse mode: gradient of a receiver misfit ====
 * The paper defines the forward leapfrog only; these calls give the exact
 * derivative of a loss of that discrete forward map (its discrete adjoint),
 * with respect to the permittivity given on a block grid (SMX_MAT_BLOCKS)
 * and to the source amplitudes.  One forward step (Sec. 4.2 / Sec. 5,
 * kick-drift-kick, S_E = K_1^{-1} M~^2_{1/eps}, S_H = K~_1^{-1} M^2_{1/mu},
 * a = dt/2):
 *   b' = b_n - a D^1 S_E d_n,  d_{n+1} = d_n + dt (D~^1 S_H b' - s_n jhat),
 *   b_{n+1} = b' - a D^1 S_E d_{n+1}.
 * Its transpose uses D~^1 = (D^1)^T, the pairing sweeps with the transposed
 * 1D factors (K_1^{-T}, K~_1^{-T}) and the symmetric masses.  FP64 contexts, and
 * SMX_MIXED_REFINED contexts, whose reverse step takes the arithmetic of their
 * forward step: each K^{-T} by FP32 sweeps with the transposed factors plus one
 * refinement with an FP64 residual, each mass apply by the FP32 kernels with FP64
 * sums (SMX_ESTATE for SMX_MIXED). */

/* Receiver points for a misfit: R maps e (N_e) to the three parametric
 * components of the discrete electric 1-form (basis of X^1_{h,0}, Sec. 2.3)
 * at n points xhat (host, n x 3, x fastest, in [0,1]); row 3 r + c.  Must be
 * called before smx_bind_workspace (the table is part of the workspace).
 * Errors: SMX_EINVAL, SMX_ESTATE (already bound or already set). */
int smx_receivers_set(smx_ctx* ctx, int n, const double* xhat);

/* out (device, 3n) = R e (device, N_e).  Errors: SMX_EINVAL (no receivers), SMX_ECUDA. */
int smx_receivers_eval(smx_ctx* ctx, const double* e, double* out);

/* ebar (device, N_e) += alpha R^T w (w device, 3n).  Errors: as smx_receivers_eval, SMX_ESTATE. */
int smx_receivers_adjoint(smx_ctx* ctx, const double* w, double alpha, double* ebar);

/* New permittivity values on the context's block grid (host, b_x b_y b_z
 * values, x fastest; field must be SMX_FIELD_D and the context created with
 * SMX_MAT_BLOCKS eps).  Updates the device Hodge tables in place (the block
 * Kronecker tile weights, or the quadrature metric scaled block by block) and
 * synchronises.  Errors: SMX_EINVAL, SMX_EMAT (value not finite and positive). */
int smx_set_material_blocks(smx_ctx* ctx, int field, const double* values);

/* One reverse step n+1 -> n.  In: the forward states d_n, d_{n+1} (device,
 * N_e), the adjoints dbar = dL/dd_{n+1} (N_e), bbar = dL/db_{n+1} (N_h);
 * ebar (device N_e or NULL): the loss's derivative with respect to e_n =
 * S_E d_n (for a misfit 1/2 dt sum |R e_n - y_n|^2: dt R^T (R e_n - y_n));
 * jhat (device N_e or NULL).  Out: dbar, bbar overwritten with dL/dd_n,
 * dL/db_n; amp_bar (device, 1 value, if jhat): dL/ds_n; eps_bar (device, one
 * value per permittivity block, or NULL): += the step's dL/deps.
 * Asynchronous on the context stream.  Errors: SMX_EINVAL (null state or
 * adjoint pointer, dt not finite and positive, eps_bar without a block
 * permittivity), SMX_ESTATE (no workspace, or an SMX_MIXED context),
 * SMX_ECUDA. */
int smx_step_adjoint(smx_ctx* ctx, const double* d_n, const double* d_np1, double* dbar, double* bbar,
                     const double* ebar, const double* jhat, double dt, double* amp_bar, double* eps_bar);

/* Start of the reverse sweep at the last step N: dbar = S_E^T ebar_N (bbar_N
 * is zero), eps_bar += the eps derivative of ebar_N^T S_E d_N.  Errors: as
 * smx_step_adjoint. */
int smx_adjoint_terminal(smx_ctx* ctx, const double* d_N, const double* ebar, double* dbar, double* eps_bar);

/* ==== Batched cavities: one persistent launch per leapfrog step ====
 * Many independent cavities (each its own bound context: any p and nel, any map
 * and material) stepped together: one cooperative launch per step runs the
 * phases of the kick-drift-kick step over a flat work list of (cavity, unit)
 * items, with grid barriers between phases.
 *   SMX_FP64 contexts: eleven phases, the same device code as smx_step (fused
 *   mass + solve passes for a star with constant material on the identity map,
 *   else a block-Kronecker or quadrature mass apply followed by the banded
 *   pairing sweeps).
 *   SMX_MIXED_REFINED contexts: twenty-five phases, the refined mixed step: FP64
 *   curls; per star an FP32 mass apply with FP64 sums, the pairing sweeps as
 *   banded FP32 recurrences, the residual of each Kronecker solve in FP64, the
 *   FP32 sweeps of the correction, and the FP64 sum (a single refined context
 *   applies dense line operators where lines are <= 80 long; the batch always
 *   runs the banded recurrences, so the two agree to the mixed tolerance, not
 *   bit for bit).
 * On a non-default stream the launches of one
 * smx_batch_step call are captured into a CUDA graph and replayed while nsteps
 * is unchanged (the step index lives in a device counter).  Each barrier wait is
 * bounded (one second); see smx_batch_status. */
typedef struct smx_batch smx_batch;

/* Build a batch over n bound contexts (host arrays; the contexts must outlive
 * the batch, stay bound to the workspaces they had here -- the batch keeps
 * their table and buffer addresses -- and share one stream, that of ctxs[0]),
 * all SMX_FP64 or all SMX_MIXED_REFINED.  Host memory only.
 * Errors: SMX_EINVAL (a context is unbound, or of another precision than
 * ctxs[0], or neither SMX_FP64 nor SMX_MIXED_REFINED), SMX_ENOMEM. */
int smx_batch_create(int n, smx_ctx* const* ctxs, smx_batch** out);
int smx_batch_destroy(smx_batch* batch);

/* Device workspace of the batch (cavity table, work lists, barrier words),
 * caller-allocated as for a context; binding uploads the work lists and picks
 * a default shape (line warps per CTA) that fits shared memory.  Binding
 * errors: SMX_EINVAL (null pointer), SMX_ESTATE (fewer bytes than
 * smx_batch_workspace_bytes, or not 256-byte aligned), SMX_ECUDA. */
int smx_batch_workspace_bytes(const smx_batch* batch, size_t* bytes);
int smx_batch_bind_workspace(smx_batch* batch, void* device_ptr, size_t bytes);

/* State of cavity i: device arrays d, b, e (consistent: e = K_1^{-1} M~ d), h
 * as for smx_step, optional source jhat with one amplitude per step in amp
 * (device), and the cavity's own dt.  Resets the step counter (amp index). */
int smx_batch_set_state(smx_batch* batch, int i, double* d, double* b, double* e, double* h, const double* jhat,
                        const double* amp, double dt);

/* nsteps leapfrog steps of every cavity: nsteps launches on the stream (one graph launch when
 * captured).  Errors: SMX_EINVAL, SMX_ESTATE (workspace not bound, or a cavity whose state was
 * never set), SMX_ECUDA. */
int smx_batch_step(smx_batch* batch, int nsteps);

/* CUDA-graph capture of smx_batch_step (default on; used on a non-default stream).  enable = 0
 * launches eagerly. */
int smx_batch_set_graphs(smx_batch* batch, int enable);

/* Synchronise; SMX_ETIMEOUT if a grid barrier gave up since the last call
 * (the results of that launch are not valid), else SMX_OK.  Once a barrier
 * has given up, every later launch returns at entry without touching the
 * state until this call clears the status and resets the barrier words. */
int smx_batch_status(smx_batch* batch);

/* Time limit of each grid-barrier wait of later launches, in seconds (default
 * 1; 0 to 60).  With 0 every wait that is not already satisfied gives up at
 * once: the tests use it to run the failure path (SMX_ETIMEOUT from
 * smx_batch_status, state of that launch invalid) without a hung GPU.
 * Errors: SMX_EINVAL. */
int smx_batch_set_wait_limit(smx_batch* batch, double seconds);

/* Autotuner: times `steps` launches for each candidate shape (1, 2, 4, 8
 * line warps per CTA, as shared memory allows) on the contexts' own state
 * vectors (zero fields; the user's state is untouched) and keeps the fastest;
 * *line_warps (optional) receives the choice. */
int smx_batch_autotune(smx_batch* batch, int steps, int* line_warps);

#ifdef __cplusplus
}
#endif

#endif /* SMX_H */
