/*
 * wfq.h -- C ABI of libwfq, the GB300 (sm_103a) implementation of the omega-FQ
 * frequency-dependent charge-response solve of arXiv 2103.00438.
 *
 * The method (Section 2.1): for N atoms at positions r_i, the complex charges q
 * at frequency w under a uniform field E0 along k solve
 *
 *     (A - z(w) I) q = R                                     (Eq. 14)
 *     A = (Kbar - P) D                                       (Eq. 17)
 *     D_ij = erf(r_ij / sqrt(w_i^2 + w_j^2)) / r_ij, D_ii = eta_i,
 *            w_i = sqrt(2/pi) / eta_i                        (Eq. 3, Eq. 4)
 *     Kbar_ij = (1 - f(r_ij)) area / r_ij, Kbar_ii = 0,
 *            f(r) = 1 / (1 + exp(-d (r / (s r0) - 1)))       (Eq. 9, Eq. 6)
 *     P = diag(sum_k Kbar_ik)                                (Eq. 16)
 *     z(w) = -(w / (2 n0 tau)) (w tau + i)                   (Eq. 12)
 *     R_i = sum_j (V_i - V_j) Kbar_ij, V_i = -E0 (r_i . k)   (Eq. 13, Eq. 2)
 *
 * The same machinery also solves the continuum (BEM) operator of Section 2.3 (Eq. 21,
 * Eq. 22), which has the same form -- a real frequency-independent matrix with a uniform
 * complex shift -- on geometries built by wfq_build_bem_geometry.
 *
 * Units are atomic units throughout (bohr, hartree, a.u. of time).
 *
 * Conventions shared by every entry point
 *   - Every function returns an int status: WFQ_OK (0) or a negative WFQ_E* code.
 *     Nothing throws across the ABI.  wfq_last_error() returns a message for the
 *     last failure on the calling thread.
 *   - The caller owns every array it passes; the library owns the handles it
 *     creates and all device memory inside them.
 *   - Complex arrays are interleaved (re, im) doubles (complex128) or floats
 *     (complex64).  A "block" of ncols complex vectors of length N is stored
 *     atom-major: element (atom i, column c) at index i * ncols + c.
 *   - Array pointers may be host or device pointers unless stated otherwise; the
 *     library tells them apart with cudaPointerGetAttributes.  Host buffers are
 *     staged through device memory inside the call.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     queued on it.  Calls that return host-visible results (solves, stats,
 *     host output buffers) synchronise that stream before returning.
 *   - One wfq_ctx per device; handles may be used from one thread at a time.
 */
#ifndef WFQ_H
#define WFQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
enum {
    WFQ_OK = 0,
    WFQ_EINVAL = -1,       /* bad argument: shape, NaN/Inf, non-positive parameter,
                              two atoms at the same position (r_ij = 0) */
    WFQ_ESINGULAR = -2,    /* omega = 0: z = 0 and A is singular (Section 2.1) */
    WFQ_ENOMEM = -3,       /* device allocation failed or the request exceeds the
                              context's memory budget */
    WFQ_ENOCONV = -4,      /* iteration limit reached; best iterate written, stats filled */
    WFQ_EBREAKDOWN = -5,   /* QMR without look-ahead met rho = 0 or sigma = 0 */
    WFQ_ETIMEOUT = -6,     /* a bounded device-side wait gave up */
    WFQ_ECUDA = -7,        /* CUDA runtime error (message in wfq_last_error) */
    WFQ_EUNSUPPORTED = -8  /* combination not available (e.g. mixed apply without the
                              bf16 D storage) */
};

typedef struct wfq_ctx wfq_ctx;
typedef struct wfq_geom wfq_geom;

/* Model parameters (atomic units).  Section 2 / Eqs. 3-12. */
typedef struct {
    double eta;        /* chemical hardness eta_i (Eq. 3 diagonal) when no per-atom array */
    double d_fermi;    /* steepness d of the Fermi damping (Eq. 6) */
    double s_fermi;    /* scale s of the Fermi damping (Eq. 6) */
    double r0;         /* equilibrium distance r0_ij (Eq. 6), uniform, bohr */
    double area;       /* effective area A_ij (Eq. 5 / Eq. 9), uniform */
    double n0;         /* electron density n0; the Drude factor is 2 n0 (Eq. 12) */
    double tau;        /* relaxation time tau (Eq. 5 / Eq. 12) */
    double cutoff_eps; /* Kbar keeps pair (i,j) iff 1 - f(r_ij) >= cutoff_eps; 0 keeps all */
} wfq_params;

/* The continuum (BEM) operator of Section 2.3 (Eq. 21, Eq. 22): a particle with the
 * Drude permittivity eps_in(w) = eps_inf - omega_p^2 / (w (w + i gamma)) in a host of
 * real permittivity eps_out.  Atomic units (hartree). */
typedef struct {
    double eps_out;    /* host permittivity, real, > 0 */
    double eps_inf;    /* background permittivity of the particle, real, > 0 */
    double omega_p;    /* plasma frequency, > 0 */
    double gamma;      /* damping rate, >= 0 */
} wfq_bem_params;

/* Storage of D chosen at geometry build (bit flags).  With no flag set D is never
 * stored: every apply recomputes its entries from the coordinates (matrix-free). */
#define WFQ_STORE_FP64   1u  /* D in FP64, N*N*8 bytes: FP64 applies and residuals */
#define WFQ_STORE_BF16X2 2u  /* D as two bf16 planes hi + lo (D ~= hi + lo), Np*Np*4 bytes
                                with Np = N rounded up to 128: the tensor-core path */
#define WFQ_STORE_F32X2  4u  /* D as two FP32 planes hi + lo (hi = fl32(D), lo = fl32(D - hi):
                                48 significant bits), N*Nq*8 bytes with Nq = N rounded up to
                                128 (512-byte rows, zero past column N): double-float products on the FP32 pipes without FP64
                                arithmetic (the shifted solver's operator, the refinement
                                residual) */
#define WFQ_STORE_F32X2_SYM 8u  /* the same FP32 hi + lo pairs for the upper triangle only
                                (D is symmetric, Eq. 3): 64 x 64 tiles (I, J), I <= J, each
                                stored row-major as 4096 hi then 4096 lo floats, tiles in
                                row order (diagonal tiles in full, zero beyond N):
                                T (T + 1) / 2 * 32 KiB with T = ceil(N / 64), about half of
                                WFQ_STORE_F32X2.  The shifted solver's D product uses it
                                when the full planes are not stored, each tile serving
                                both D_IJ x_J and D_IJ^T x_I (about the same time, half
                                the memory). */

/* Arithmetic of an apply / of the inner Krylov iterations. */
enum {
    WFQ_PREC_FP64 = 0,     /* FP64 operator, complex128 vectors */
    WFQ_PREC_MIXED = 1,    /* D.x from 3 bf16 products (hi.hi + hi.lo + lo.hi) with FP32
                              accumulation on the tensor cores, D from the stored bf16 planes
                              or generated from the coordinates -- or, without stored planes
                              and after wfq_fmm_build, by the fast multipole method (as
                              WFQ_PREC_FMM, up to 256 columns per product); complex64
                              vectors; solves add iterative refinement on top, whose true
                              residuals use the WFQ_PREC_DF product (on a geometry with no
                              stored D, D regenerated in FP64 once that product's rounding
                              holds a residual at a floor) */
    WFQ_PREC_DF = 2,       /* wfq_apply and the refinement residuals: complex128 vectors, D.x
                              with float-pair operands and double-float accumulation (~2^-48
                              relative per product) on the FP32 pipes: D split from the stored
                              FP64 D (up to 4 columns: the FP64 GEMV), or read from the stored
                              FP32 pair planes or symmetric tiles, or regenerated from the
                              coordinates in double-float (near pairs in FP64) */
    WFQ_PREC_FMM = 3       /* wfq_apply only: complex64 vectors, D.x by the fast multipole
                              method built with wfq_fmm_build (near field by Eq. 3, far field
                              1/r by Chebyshev interpolation), FP32 arithmetic */
};

/* Per-solve statistics. */
typedef struct {
    int32_t iters;        /* operator applications inside Krylov iterations */
    int32_t restarts;     /* restart cycles after the first (GMRES) */
    int32_t refinements;  /* FP64 true-residual evaluations after the first cycle */
    int32_t status;       /* WFQ_OK, WFQ_ENOCONV or WFQ_EBREAKDOWN */
    double rel_residual;  /* ||R - (A - zI) q||_2 / ||R||_2, FP64 (Eq. 27 / ||R||) */
    double rmse;          /* ||R - (A - zI) q||_2 / sqrt(N)  (Eq. 33) */
} wfq_stats;

/* ---------------------------------------------------------------- context */

/* Creates a context on CUDA device `device`.  *ctx is set on success. */
int wfq_create(wfq_ctx **ctx, int device);

/* Releases the context.  Geometries created on it must be freed first. */
int wfq_destroy(wfq_ctx *ctx);

/* Message of the last failure on this thread ("" if none).  Owned by the library. */
const char *wfq_last_error(void);

/* Number of CUDA kernels libwfq has launched in this process so far (all threads).
 * Profiling aid: the difference across a region counts the library's launches in it. */
int64_t wfq_kernel_launches(void);

/* Device-memory accounting (a deployment aid; the paper has no counterpart).
 * out[0]: device allocations the library has requested in this process so far (all
 * contexts, all threads; pool and plain allocations); out[1]: bytes the context's
 * stream-ordered pool holds reserved; out[2]: bytes of it in use now; out[3]: the
 * pool's in-use high-water mark.  out: host, 4 values, caller-owned. */
int wfq_memory_stats(wfq_ctx *ctx, int64_t *out);

/* Kernel timing (profiling aid).  While enabled, the library records a pair of CUDA
 * events on the launching stream around every launch of the kernels below;
 * wfq_profile_read synchronises those events and returns the launch count and the
 * summed device time since the last wfq_profile(ctx, 1) call. */
enum {
    WFQ_KT_GEMM_MIXED = 0,   /* 3xBF16 tensor-core GEMM  U = D X   (mixed apply) */
    WFQ_KT_DAPPLY_FP64 = 1,  /* FP64 dense product U = D X (stored or recomputed D) */
    WFQ_KT_SPARSE = 2,       /* sparse term and shift  Y = Kbar U - P U - z X */
    WFQ_KT_ORTHO = 3,        /* Arnoldi orthogonalisation of one GMRES step (projections,
                                norm, Givens, scaling) / the vector updates of a QMR step */
    WFQ_KT_RESIDUAL = 4,     /* FP64 true residual of a cycle (gathers, product, norms) */
    WFQ_KT_DGEMV_DF = 5,     /* shifted GMRES: double-float D product of the real Arnoldi
                                vectors (one launch per group of <= 4 directions) */
    WFQ_KT_FMM = 6,          /* the fast-multipole D product (all its passes) */
    WFQ_KT_COUNT = 7
};

/* enable != 0: reset the counters and start recording; enable == 0: stop. */
int wfq_profile(wfq_ctx *ctx, int enable);

/* Launches, summed device milliseconds and summed work of kernel class `kind` (WFQ_KT_*).
 * Work: WFQ_KT_GEMM_MIXED -- tensor flops of the three bf16 products, 6 N^2 C per launch
 * (C = real columns of that launch); WFQ_KT_DAPPLY_FP64 -- 2 N^2 C flops; WFQ_KT_DGEMV_DF --
 * algorithmic bytes of D read, 8 N^2 (the entries; padding columns not counted); WFQ_KT_FMM
 * -- N^2, the pair interactions the product stands for; others 0.
 * Any out-pointer may be NULL. */
int wfq_profile_read(wfq_ctx *ctx, int kind, int64_t *launches, double *total_ms, double *work);

/* ---------------------------------------------------------------- geometry */

/* Builds everything that depends only on the structure (Section 2.1: A and R do
 * not depend on omega):
 *   - per-atom data (positions, Gaussian widths from Eq. 4),
 *   - Kbar as CSR with a cell-list neighbour search (pairs with
 *     1 - f(r) >= cutoff_eps, Eq. 9) and P (Eq. 16),
 *   - D (Eq. 3) in the storages requested by `store` (WFQ_STORE_* flags).
 * xyz: host, n x 3 row-major bohr.  eta: host array of n hardnesses or NULL (then
 * p->eta for every atom).  Fails with WFQ_EINVAL for n < 1, non-finite input,
 * non-positive eta/d/s/r0/area/n0/tau, cutoff_eps outside [0, 1), or two atoms
 * closer than 1e-8 bohr.  *out is set on success. */
int wfq_build_geometry(wfq_ctx *ctx, int64_t n, const double *xyz, const double *eta,
                       const wfq_params *p, uint32_t store, wfq_geom **out);

/* Builds a geometry for the continuum BEM operator of Section 2.3 (the comparison with
 * continuum approaches), which has the same algebraic form as the omega-FQ system: a real
 * frequency-independent matrix with a uniform complex shift.  Eq. 21,
 * (Lambda(w) I + F) sigma = -dphi/dn with Lambda(w) = 2 pi (eps_out + eps_in(w)) /
 * (eps_out - eps_in(w)) and F_ij = n_i . (r_i - r_j) / |r_i - r_j|^3 (Eq. 22), is
 * discretised by collocation at n surface elements and solved as (A - zI) q = R for the
 * element charges q_i = a_i sigma_i:
 *     A_ij = a_i n_i . (r_i - r_j) / |r_i - r_j|^3  (i != j),
 *     A_ii = H_i sqrt(pi a_i)  (Eq. 22's principal value over the element itself, taken
 *            as a flat disk of area a_i on a surface of mean curvature H_i),
 *     z(w) = -Lambda(w),   R_i = -E0 a_i (n_i . k)  (the field phi = -E0 k . r; the sign
 *            is the one for which q is the physical charge: the printed right-hand side
 *            -dphi/dn gives -q).
 * The polarizability (wfq_polarizability) is then sum_i q_i r_i / E0 as for omega-FQ.
 * xyz: host n x 3 collocation points (bohr); normal: host n x 3 outward unit normals
 * (norm within 1e-6 of 1); area: host n element areas (> 0); curvature: host n mean
 * curvatures H_i (1 / bohr, positive where the surface bends away from its outward normal,
 * as on a sphere), or NULL for flat elements (H = 0).  store: must include WFQ_STORE_FP64;
 * WFQ_STORE_F32X2 (the shifted solver's fastest operator) and WFQ_STORE_BF16X2 (needed by
 * WFQ_PREC_MIXED) are optional; WFQ_STORE_F32X2_SYM is rejected (A is not symmetric).
 * Operator entries are never regenerated from the coordinates (no matrix-free path).
 * Every entry point that takes a geometry accepts a BEM geometry, with these differences:
 * wfq_apply computes y = A x - z x; wfq_rhs returns the R above; wfq_solve_qmr returns
 * WFQ_EUNSUPPORTED (its J-symmetry needs A = (Kbar - P) D with D symmetric);
 * WFQ_PREC_MIXED without WFQ_STORE_BF16X2 and wfq_apply_mixed_noalloc return
 * WFQ_EUNSUPPORTED; a frequency at which eps_in = eps_out (Lambda infinite) is WFQ_EINVAL,
 * omega = 0 WFQ_ESINGULAR.  Fails with WFQ_EINVAL for n < 1, non-finite input, a
 * non-positive area or parameter, a normal that is not a unit vector, or two elements
 * closer than 1e-8 bohr.  *out is set on success. */
int wfq_build_bem_geometry(wfq_ctx *ctx, int64_t n, const double *xyz, const double *normal,
                           const double *area, const double *curvature, const wfq_bem_params *p,
                           uint32_t store, wfq_geom **out);

int wfq_free_geometry(wfq_geom *g);

/* n: atoms; nnz: stored Kbar pairs; device_bytes: device memory held by g. */
int wfq_geometry_info(const wfq_geom *g, int64_t *n, int64_t *nnz, int64_t *device_bytes);

/* ---------------------------------------------------------------- operator */

/* y = (A - z(omega_c) I) x for ncplx complex columns (Eq. 14's operator, applied
 * through the factored form of Eq. 17):  u = D x,  y = Kbar u - P u - z x.
 * omega: host array of ncplx frequencies (hartree), one per column; omega_c = 0 is
 * allowed here (z = 0).  x, y: N x ncplx atom-major blocks, complex128 for
 * WFQ_PREC_FP64 / WFQ_PREC_DF and complex64 for WFQ_PREC_MIXED; x and y must not overlap.
 * FP64 / DF use the stored FP64 D if present, else recompute D (matrix-free).  MIXED uses
 * the stored bf16 planes if present, else generates the D tiles from the coordinates on
 * the fly (matrix-free tensor-core path).  Asynchronous on `stream` when x and y are
 * device pointers. */
int wfq_apply(wfq_geom *g, int64_t ncplx, const double *omega, const void *x, void *y,
              int prec, void *stream);

/* Allocation-free variant of wfq_apply with WFQ_PREC_MIXED (the paper has no
 * counterpart: this is a deployment facility).  It is for callers that must not
 * allocate device memory during the apply -- code that runs inside a fixed memory
 * budget or arena, or in a context where cudaMalloc is not allowed or would stall the
 * device -- and it computes exactly what wfq_apply(..., WFQ_PREC_MIXED, ...) computes
 * with the same kernels.
 *   - x, y: DEVICE pointers of the context's device, N x ncplx complex64 atom-major
 *     (host pointers and other devices' pointers are rejected with WFQ_EINVAL, since
 *     staging them would allocate).  omega: host, ncplx values, read during the call
 *     and handed to the device as a kernel argument (no copy of the caller's array), so
 *     ncplx <= 1024.  The caller still owns and passes all inputs and outputs.
 *   - Scratch (the bf16 planes of x, u = D x and the shifts) lives in one static
 *     32 MiB device array that every device which loads the library keeps until the
 *     process exits.  A call needs
 *         4*ceil32(2*ncplx)*ceil128(N) + align256(8*N*ncplx) + align256(16*ncplx)
 *     bytes of it (ceilK: rounded up to a multiple of K; align256: to 256 bytes); a
 *     call needing more than 32 MiB fails with WFQ_EINVAL and a message; use wfq_apply
 *     then.
 *   - The first call on a device looks up the array's device address (once per
 *     device, with that device current); make that first call before any stream
 *     capture.
 *   - All calls share the one array and every call overwrites what it reads, so no
 *     clearing is needed; calls whose work overlaps on the GPU (different streams,
 *     threads or devices' streams without ordering) race on it and must be
 *     serialised by the caller.
 *   - Needs WFQ_STORE_BF16X2 (else WFQ_EUNSUPPORTED).  No device memory is allocated
 *     or freed by this call. */
int wfq_apply_mixed_noalloc(wfq_geom *g, int64_t ncplx, const double *omega, const void *x,
                            void *y, void *stream);

/* Far-field-compressed D product (the fast multipole method the paper's conclusions name
 * as the way past the O(N^2) matrix-vector product; the paper gives no FMM of its own):
 * builds, for an omega-FQ geometry, the tree and operators that wfq_apply(...,
 * WFQ_PREC_FMM, ...) uses.  The method is the Chebyshev-interpolation FMM of Fong and
 * Darve: a uniform tree over the bounding cube (a quadtree over the bounding square when
 * all atoms share one z), as deep as leaves of side >= 6 max_ij sqrt(w_i^2 + w_j^2) allow
 * (so every far pair has erf(r / s_ij) = 1 in FP64 and D_ij = 1 / r_ij exactly, Eq. 3);
 * pairs in the same or adjacent leaves by Eq. 3; all other pairs through `order`
 * Chebyshev nodes per dimension per box (P2M, M2M, M2L over interaction lists, L2L,
 * L2P).  The far field's relative error falls geometrically with order (about 1e-6 of
 * sum_j |D_ij x_j| at order 6 on a flat flake).  order: 2..16 for a flat structure, 2..6
 * for a 3D one.  wfq_apply with WFQ_PREC_FMM takes at most 256 complex columns per call.
 * Host work O(N log N) plus
 * the operator tables (order^(2 dim) floats per offset); device memory is counted in the
 * geometry's bytes and freed with it; a second call replaces the first.  WFQ_EUNSUPPORTED
 * for BEM geometries, WFQ_EINVAL for an order out of range. */
int wfq_fmm_build(wfq_geom *g, int order);

/* The tree of wfq_fmm_build: out[0] dimension (2: quadtree, 3: octree), out[1] depth,
 * out[2] order, out[3] non-empty leaves, out[4] non-empty boxes of all levels, out[5]
 * interaction-list entries, out[6] near-list entries.  WFQ_EUNSUPPORTED if not built. */
int wfq_fmm_info(const wfq_geom *g, int64_t *out);

/* Right-hand sides R (Eq. 13 with the potential of Eq. 2) for ndir field
 * directions.  dirs: host, ndir x 3 (need not be unit vectors; the field is E0 * dir).
 * R: N x ndir atom-major real (FP64). */
int wfq_rhs(wfq_geom *g, int ndir, const double *dirs, double E0, double *R, void *stream);

/* ---------------------------------------------------------------- solvers */

/* Solves (A - z(omega_f) I) q = R(dir_d) for every frequency f < nfreq and field
 * direction d < ndir at once (ncols = nfreq * ndir complex columns sharing D and
 * Kbar; column c = f * ndir + d), by GMRES (Section 3, Eq. 24) from q0 = 0.
 *   m: restart length (GMRES(m)); 0 = unrestarted (one cycle of up to max_iter).
 *   rel_tol: stop when the FP64 true residual satisfies ||R - (A - zI) q|| <= rel_tol ||R||
 *            for every column (Eq. 27 relative to ||R||).
 *   max_iter: cap on Krylov iterations per column.
 *   prec: WFQ_PREC_FP64 -- FP64 operator and complex128 Krylov basis;
 *         WFQ_PREC_MIXED -- each restart cycle iterates with the mixed operator and a
 *         complex64 basis (FP64-grade inner products, FP64 norms and Givens rotations);
 *         a cycle starts from the true residual at FP64 accuracy (iterative refinement)
 *         -- or, while every column is still above 1e-3 ||R||, from the mixed-operator
 *         residual.  A column is finished by plain FP64 GMRES(m) from its iterate when its
 *         true residual shrank by less than 2x in each of two consecutive cycles while the
 *         inner solve reached its own target (the mixed operator's residual estimate below
 *         a quarter of the true residual: a precision floor), or in each of 20 consecutive
 *         cycles otherwise.  The true residuals use double-float D products (stored float
 *         pairs, else D regenerated per product); on a geometry with no stored D whose
 *         regenerated residual reaches such a floor, the residuals switch to D regenerated
 *         in FP64 and the column stays in mixed precision.
 *         Convergence is always decided on the FP64-accuracy true residual (FP64 solves:
 *         FP64 D products in the residual; their Arnoldi products on a geometry without
 *         an FP64 D are the double-float ones).
 * With the environment variable WFQ_TRACE set (not "0"), the solvers print one line per
 * restart cycle (active and escalated columns, steps, worst true residual) on stderr.
 * q: output, N x ncols complex128 atom-major.  stats: host array of ncols, or NULL.
 * Returns WFQ_OK when every column converged, WFQ_ENOCONV otherwise (q holds the last
 * iterate), WFQ_ESINGULAR if some omega is 0.  Synchronises `stream`. */
int wfq_solve_gmres(wfq_geom *g, int64_t nfreq, const double *omega, int ndir,
                    const double *dirs, double E0, int m, double rel_tol, int max_iter,
                    int prec, double *q, wfq_stats *stats, void *stream);

/* As wfq_solve_gmres, by shifted GMRES: A = (Kbar - P) D and R are real and do not
 * depend on omega (Section 2.1), so the Krylov space of A - z(omega) I from R is the
 * same for every frequency.  One real Arnoldi process per field direction (FP64 basis,
 * D applied with double-float products) serves all nfreq frequencies; each column's
 * GMRES iterate (Eq. 24, q0 = 0) comes from its own complex Givens QR of the shared
 * Hessenberg matrix shifted by z(omega).  One D product of ndir real vectors per
 * iteration instead of one of 2 * nfreq * ndir.
 *   m_max: cap on the Arnoldi basis (0 = 600 vectors; memory 8 * N * ndir * (m_max + 1)
 *          bytes plus 16 * m_max^2 / 2 per column).
 *   prec: precision of the block GMRES(50) that continues, from their iterate, the
 *         columns whose FP64 true residual is still above rel_tol at the end (basis cap
 *         reached, or rounding of the shared process): WFQ_PREC_MIXED or WFQ_PREC_FP64.
 * D comes from the FP32 pair planes (WFQ_STORE_F32X2, fastest), the symmetric tiles
 * (WFQ_STORE_F32X2_SYM), the FP64 D, or -- with none of them stored -- is regenerated from
 * the coordinates in double-float for every product (near pairs in FP64; matrix-free).
 * stats: iters = Arnoldi steps the column used plus any continuation's; restarts = 1 +
 * the continuation's when a column was continued.  Other arguments and results as
 * wfq_solve_gmres. */
int wfq_solve_gmres_shifted(wfq_geom *g, int64_t nfreq, const double *omega, int ndir,
                            const double *dirs, double E0, int m_max, double rel_tol,
                            int max_iter, int prec, double *q, wfq_stats *stats, void *stream);

/* As wfq_solve_gmres, with the J-symmetric QMR-from-BCG method without look-ahead
 * (Section 3; J = D since D A = A^T D, Eq. 18).  The bilinear form u^T D v needs D v,
 * which the operator apply already produces, so each iteration costs one D product.
 * With WFQ_PREC_MIXED the QMR recurrence restarts from the FP64 true residual every
 * `refine_every` iterations (0 = when its own residual estimate converges, at the latest
 * after 300 iterations); a column whose recurrence broke down, or whose true residual
 * shrank by less than 2x in two consecutive restarts after each of which the inner QMR had
 * converged (in 20 consecutive restarts otherwise), is finished by plain FP64 GMRES(50) from
 * its iterate; the residual switch of a matrix-free geometry is as in wfq_solve_gmres.
 * Returns WFQ_EBREAKDOWN if rho or sigma vanishes in some column of an FP64 solve. */
int wfq_solve_qmr(wfq_geom *g, int64_t nfreq, const double *omega, int ndir,
                  const double *dirs, double E0, double rel_tol, int max_iter, int prec,
                  int refine_every, double *q, wfq_stats *stats, void *stream);

/* Complex polarizability of each solved column: alpha[c][k'] = sum_i q_i r_{i,k'} / E0
 * for k' = x, y, z (Section 4.1, Eq. 28: sigma_k = (4 pi w / c) Im alpha_kk).
 * q: N x ncols complex128 (host or device).  alpha: host, ncols x 3 complex128. */
int wfq_polarizability(wfq_geom *g, int64_t ncols, const double *q, double E0,
                       double *alpha, void *stream);

/* Cross sections of solved columns (Section 4.1): the longitudinal cross section of
 * Eq. 28, sigma_k(w) = (4 pi w / c) sum_i (k_i / E0) Im q_i^k, for each column
 * c = f * ndir + d, with k = dirs[d] / |dirs[d]| and the field amplitude E0 |dirs[d]|
 * (the field the solvers apply for that direction), i.e.
 *     sigma[c] = (4 pi omega[f] / c) Im(dirs[d] . alpha_c) / |dirs[d]|^2,
 * alpha_c of wfq_polarizability; and, when sigma_iso is not NULL, the mean over the
 * ndir directions per frequency -- the isotropic cross section of Eq. 29 when the
 * directions are x, y, z (any orthonormal triad).  c = 137.035999084 (atomic units).
 *   omega: host, nfreq values (hartree); dirs: host, ndir x 3 (non-zero, finite).
 *   q: N x (nfreq * ndir) complex128, host or device (the solvers' output layout).
 *   sigma: nfreq x ndir FP64 (bohr^2), sigma_iso: nfreq FP64 or NULL; host or device.
 * Blocks until the results are written.  WFQ_EINVAL on NULL, empty, non-finite or
 * zero-length arguments. */
int wfq_cross_section(wfq_geom *g, int64_t nfreq, const double *omega, int ndir, const double *dirs,
                      double E0, const double *q, double *sigma, double *sigma_iso, void *stream);

/* ---------------------------------------------------------------- serving */

/* A request server on one context: `nworkers` threads, each with its own CUDA stream,
 * take solve requests from a FIFO queue.  Structures stay resident (requests reference
 * geometries built with wfq_build_geometry; a geometry must outlive its requests).
 * A worker that becomes free takes the oldest request whose batch fits the memory budget
 * and merges into the same block solve every queued request on the same geometry with
 * the same settings (continuous batching), up to max_columns complex columns; batches on
 * different workers run concurrently.  A batch on a geometry with a stored D
 * (WFQ_STORE_F32X2 or WFQ_STORE_FP64) is solved by shifted GMRES (as
 * wfq_solve_gmres_shifted: one real Arnoldi process per distinct field direction of the
 * batch for all its frequencies; m is not used, continuations run GMRES(50)); otherwise
 * by mixed-precision GMRES(m) with FP64 refinement (as wfq_solve_gmres with
 * WFQ_PREC_MIXED).  BEM geometries (wfq_build_bem_geometry, which always store the FP64
 * operator) take the shifted path; their continuations run in FP64 unless the bf16 planes
 * are stored too.
 *   budget_bytes: device memory for the structures in use plus the batches in flight:
 *   a batch starts only while the device bytes of every geometry with requests queued or
 *   running (wfq_geometry_info's device_bytes), the footprints of the batches in flight (Krylov
 *   bases, blocks, scratch) and its own footprint fit in it; otherwise it waits until
 *   running batches finish.  A batch still runs when nothing else is in flight. */
typedef struct wfq_server wfq_server;
int wfq_server_create(wfq_ctx *ctx, int nworkers, int64_t budget_bytes, int max_columns,
                      wfq_server **out);

/* Queues one request: nfreq frequencies x ndir directions (columns c = f * ndir + d, as in
 * wfq_solve_gmres).  q_host (N x ncols complex128) and stats (ncols, or NULL) are host
 * buffers the caller keeps valid until the request is complete; the server writes them.
 * Returns at once with *request_id.  WFQ_ENOMEM if the request's footprint plus its
 * geometry's device bytes cannot fit the budget,
 * WFQ_ESINGULAR for omega = 0. */
int wfq_server_submit(wfq_server *s, wfq_geom *g, int64_t nfreq, const double *omega, int ndir,
                      const double *dirs, double E0, int m, double rel_tol, int max_iter,
                      double *q_host, wfq_stats *stats, int64_t *request_id);

/* State of a request; wait != 0 blocks until it is complete.  When complete: status
 * (WFQ_OK, WFQ_ENOCONV or an error), latency_s (submit -> completion), queue_s (submit ->
 * start of its batch), batch_columns (columns of the block solve it ran in), and the
 * request is released (its id becomes unknown).  Any out-pointer may be NULL. */
int wfq_server_poll(wfq_server *s, int64_t request_id, int wait, int *done, int *status,
                    double *latency_s, double *queue_s, int *batch_columns);

/* Finishes every queued request, then stops the workers and frees the server. */
int wfq_server_destroy(wfq_server *s);

#ifdef __cplusplus
}
#endif

#endif /* WFQ_H */
