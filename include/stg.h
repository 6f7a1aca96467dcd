/*
 * stg.h -- C ABI of the GB300 staggered-fermion hot path.
 *
 * Operations (arXiv:1801.01473):
 *   - the off-diagonal blocks D_eo / D_oe of the staggered Dirac matrix (Sec. 2),
 *     with the staggered and antiperiodic-time phases attached to the links as
 *     u_mu(x) U_mu(x) (Sec. 4.1) and optional 12-real link compression
 *     r3 = (r1 x r2)^* (Sec. 4.1);
 *   - the shifted normal operator  A_sigma = m^2 + sigma - D_eo D_oe  (Eq. shift_eo);
 *   - the multi-shift CG solve of A_sigma_i x_i = b for all poles sigma_i (Sec. 2);
 *   - the fermion force of S = sum_i r_i Re(b^dag x_i) with respect to the links;
 *   - the k-times stout smearing of the links that D uses, and the chain rule that maps a
 *     force on the smeared links back to the unsmeared ones (Sec. 2-3);
 *   - the tree-level Symanzik gauge action and its force (Sec. 2-3).
 *
 * Conventions.
 *   site      i = x + Lx*(y + Ly*(z + Lz*t)), mu = 0..3 = x, y, z, t; all extents even.
 *   parity    (x+y+z+t) mod 2; a site of either parity has half index i>>1 (Vh = V/2).
 *   phases    u_mu(x) = (-1)^(x_0+...+x_{mu-1}), times -1 on t-links with x_t = Lt-1
 *             when the lattice is antiperiodic in time.
 *   operator  (D psi)(x) = 1/2 sum_mu [ u_mu(x) U_mu(x) psi(x+mu) - u_mu(x-mu) U_mu(x-mu)^dag psi(x-mu) ].
 *             D_eo maps odd -> even, D_oe maps even -> odd; D_oe^dag = -D_eo.
 *
 * Canonical (interchange) layouts, complex128, row-major:
 *   links     [4][Lt][Lz][Ly][Lx][3][3]           (U[mu][i][a][b], a = row)
 *   fields    [Vh][3] on one parity, half-index order
 *   force     [4][Lt][Lz][Ly][Lx][3][3]
 * Internal layouts (what stg_dslash_* and stg_normal_op read and write):
 *   F64 field: 3 arrays of Vh double2 (colour-major structure of arrays), 48 B/site.
 *   F32 field: Vh float4 (colours 0,1) followed by Vh float2 (colour 2), 24 B/site.
 *   DS field:  3 arrays of Vh float4 (re.hi, re.lo, im.hi, im.lo), 48 B/site.
 *   A gauge of precision F64 works on F64 fields, DS on DS fields; F32, BF16 and F16 gauges
 *   work on F32 fields.
 *
 * Memory.  Every pointer argument named *_dev is device memory owned by the caller
 * and must stay valid until the work queued on `stream` has finished.  Host arrays are
 * read before the call returns.  `stream` is a cudaStream_t (NULL = legacy default stream).
 * Opaque handles (stg_lattice, stg_gauge) and the solver workspaces are owned by the
 * library; *_destroy releases them.
 *
 * Errors.  Every call returns stg_status; nothing aborts or exits.  Arguments are
 * checked on the host before any launch.  stg_last_error() returns a message describing
 * the last failure of the calling thread.  Calls are asynchronous on `stream` except the
 * solvers, which synchronise the stream to fill their statistics.
 */
#ifndef STG_H
#define STG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    STG_OK = 0,
    STG_ERR_ARG = -1,     /* null pointer, bad enum, bad count, misaligned pointer          */
    STG_ERR_SHAPE = -2,   /* lattice extents not even / too small, mismatched lattices      */
    STG_ERR_CUDA = -3,    /* a CUDA runtime call failed (message in stg_last_error)          */
    STG_ERR_NOCONV = -4,  /* solver hit max_iter; statistics filled, best iterate returned   */
    STG_ERR_TIMEOUT = -5, /* a bounded device-side wait gave up                              */
    STG_ERR_OOM = -6      /* device allocation failed                                       */
} stg_status;

/* STG_DS: "double-single" storage, every real number as a pair of floats hi + lo (48-bit
 * significand, relative rounding ~2^-47), computed with error-free FP32 transformations:
 * FP64-class accuracy on the FP32 pipes.  Same bytes as F64. */
typedef enum { STG_F64 = 0, STG_F32 = 1, STG_BF16 = 2, STG_F16 = 3, STG_DS = 4 } stg_prec;
typedef enum { STG_RECON18 = 18, STG_RECON12 = 12 } stg_recon;

typedef struct stg_lattice stg_lattice;
typedef struct stg_gauge stg_gauge;

/* Human-readable name of a status code; never NULL. */
const char *stg_status_string(stg_status s);
/* Message of the last failing call on this thread ("" if none); never NULL. */
const char *stg_last_error(void);
/* Library version string. */
const char *stg_version(void);

/* ---- lattice geometry ---------------------------------------------------------------- */

/* dims = {Lx, Ly, Lz, Lt}; every extent even and >= 2, V <= 2^31.  t_antiperiodic != 0
 * puts the antiperiodic boundary sign on the t-links with x_t = Lt-1 (Sec. 4.1 folds it
 * into u_mu).  *out receives a new handle.  STG_ERR_SHAPE on odd or small extents. */
stg_status stg_lattice_create(const int32_t dims[4], int32_t t_antiperiodic, stg_lattice **out);
void stg_lattice_destroy(stg_lattice *lat);
/* Number of sites of one parity (0 even, 1 odd) or of the whole lattice (-1); -1 on NULL.
 * The even/odd split is that of Eq. shift_eo (Sec. 2): fields live on one parity, each of
 * V/2 sites (Sec. 4.1 stores them the same way). */
int64_t stg_lattice_sites(const stg_lattice *lat, int32_t parity);

/* ---- gauge field ----------------------------------------------------------------------- */

/* Copies the canonical complex128 links (device memory, [4][V][3][3]) into a
 * library-owned copy in the internal structure-of-arrays layout
 * [mu][parity][chunk][Vh] at precision `prec`.  recon = STG_RECON12 keeps only rows 1 and
 * 2 and rebuilds row 3 = (r1 x r2)^* in registers (Sec. 4.1); this is exact only for
 * SU(3) links.  BF16/F16 require STG_RECON12.  The copy is finished when the work on
 * `stream` is.  The lattice must outlive the gauge. */
stg_status stg_gauge_create(const stg_lattice *lat, const void *links_c128_dev, stg_prec prec, stg_recon recon,
                            void *stream, stg_gauge **out);
/* As stg_gauge_create, with a U(1) phase field: theta_dev (device, FP64, canonical [4][V], radians)
 * gives every link the phase u = exp(i theta_mu(x)) on top of the staggered and boundary signs,
 * so that D uses exp(i theta) U forward and exp(-i theta) U^dag backward (Sec. 4.1: imaginary
 * chemical potential and background fields as a per-flavour U(1) field).  The phases are stored
 * beside the links: as float angles turned into cos + i sin on line for F32/BF16/F16 links (the
 * paper's choice for memory-bound operators), as precomputed (cos, sin) double pairs for F64 and
 * DS links (FP64 trigonometry is expensive on GB300); 12-real compression applies to the SU(3)
 * part only.  Every operation
 * accepts such a gauge; the solvers need the inner gauge to carry the same phases. */
stg_status stg_gauge_create_u1(const stg_lattice *lat, const void *links_c128_dev, const double *theta_dev,
                               stg_prec prec, stg_recon recon, void *stream, stg_gauge **out);
/* Replaces the links of an existing gauge (same lattice, precision, compression) with new ones,
 * without allocating: the MD evolution changes the links every step (Sec. 3), and a production
 * loop keeps one gauge per precision and refreshes it.  theta_dev must be given (device, FP64,
 * [4][V]) exactly when the gauge was created with stg_gauge_create_u1, NULL otherwise.  The
 * double-single and FP32 companions that solves and forces created for an F64 gauge are refreshed
 * too.  Stream-ordered: work already queued on `stream` sees the old links, later work the new;
 * the gauge may not be in use on another stream meanwhile.  STG_ERR_ARG on null, misaligned or
 * mismatched arguments. */
stg_status stg_gauge_update(stg_gauge *g, const void *links_c128_dev, const double *theta_dev, void *stream);
void stg_gauge_destroy(stg_gauge *g);
/* Bytes of the internal link copy (4 V links). */
size_t stg_gauge_bytes(const stg_gauge *g);

/* ---- fermion fields ----------------------------------------------------------------------- */

/* Bytes of one parity's field in the internal layout for vector precision F64, DS or F32
 * (48, 48 or 24 bytes per site); 0 for any other precision or a NULL lattice.  The internal
 * layout is a structure of arrays over the sites of one parity (Sec. 4.1's colour-vector
 * layout, one array per colour component, so that consecutive threads read consecutive
 * addresses); 48 bytes per site is the paper's FP64 figure for one colour vector (Sec. 3.1). */
size_t stg_field_bytes(const stg_lattice *lat, stg_prec vec_prec);
/* canonical complex128 [Vh][3] (device) <-> internal layout (device). vec_prec F64, DS or F32.
 * The conversion between the array-of-structures interchange layout and the structure-of-arrays
 * layout of Sec. 4.1 (see stg_field_bytes); F32 and DS round each FP64 component (to nearest,
 * DS keeping the rounding error in its second float).  STG_ERR_ARG on NULL pointers or another
 * precision; asynchronous on `stream`. */
stg_status stg_field_pack(const stg_lattice *lat, stg_prec vec_prec, const void *canon_c128_dev, void *internal_dev,
                          void *stream);
stg_status stg_field_unpack(const stg_lattice *lat, stg_prec vec_prec, const void *internal_dev, void *canon_c128_dev,
                            void *stream);

/* ---- the staggered operator (Sec. 2, Sec. 4.2) ----------------------------------------------- */

/* out_even = D_eo in_odd.  Internal layout at the gauge's vector precision. in/out must not
 * overlap.  Pointers 16-byte aligned. */
stg_status stg_dslash_eo(const stg_gauge *g, void *out_even_dev, const void *in_odd_dev, void *stream);
/* out_odd = D_oe in_even. */
stg_status stg_dslash_oe(const stg_gauge *g, void *out_odd_dev, const void *in_even_dev, void *stream);
/* out_parity 0: out = D_eo in (as stg_dslash_eo); 1: out = D_oe in (as stg_dslash_oe).
 * STG_ERR_ARG for any other out_parity. */
stg_status stg_dslash(const stg_gauge *g, int32_t out_parity, void *out_dev, const void *in_dev, void *stream);
/* nrhs applications of one block sharing each link load: out_parity 0 -> D_eo, 1 -> D_oe;
 * field j at in_dev + j*stride_bytes (same for out).  1 <= nrhs <= 64; stride a multiple of
 * 16 bytes and >= stg_field_bytes. */
stg_status stg_dslash_multi(const stg_gauge *g, int32_t out_parity, int32_t nrhs, void *out_dev, const void *in_dev,
                            size_t stride_bytes, void *stream);

/* D_eo (out_parity 0) or D_oe (1) of nfield canonical [Vh][3] fields that live in HOST memory,
 * complex128 (host_prec STG_F64) or complex64 (STG_F32: half the bytes over the host link, for
 * gauges that compute in FP32 anyway): out_host[k] = D in_host[k].  A three-stage pipeline on internal streams overlaps the
 * host->device copy of field k+1, pack / D / unpack of field k (the gauge's precision) and the
 * device->host copy of field k-1, with two device staging slots per stage (4 canonical + 4 internal
 * fields of device memory, allocated and freed by the call).  Host buffers should be pinned for the
 * copies to overlap.  Ordered after the work queued on `stream`; returns when every output is in
 * host memory.  No in/out aliasing. */
stg_status stg_dslash_host(const stg_gauge *g, int32_t out_parity, stg_prec host_prec, int32_t nfield,
                           const void *const *in_host, void *const *out_host, void *stream);

/* out_even = (m^2 + shift) in_even - D_eo D_oe in_even  (Eq. shift_eo), tmp_odd a caller buffer
 * of stg_field_bytes.  If pq_dev != NULL, *pq_dev (one device double) receives Re<in, out>,
 * reduced in FP64 in a fixed order.  The reduction uses a scratch buffer owned by the gauge
 * handle: concurrent stg_normal_op calls on one gauge in different streams race on it. */
stg_status stg_normal_op(const stg_gauge *g, double mass, double shift, void *out_even_dev, const void *in_even_dev,
                         void *tmp_odd_dev, double *pq_dev, void *stream);

/* Same operation and results as stg_normal_op with pq_dev, for callers that cannot allocate
 * device memory when they call it: a host framework that owns all device memory through its own
 * pool, or a time-stepping loop that must not call cudaMalloc/cudaFree (they can synchronize the
 * device, or fail once memory is partitioned).  It needs no tmp_odd: the odd temporary and the
 * partial sums live in one 32 MiB file-scope __device__ array that every GPU loading the library
 * holds until exit.  The paper has no counterpart of this entry point.
 *   Limit: Vh <= 697232 sites per parity for F64 and DS (double-single) gauges, whose odd
 *          temporary takes 48 B per site, and <= 1390848 for F32/BF16/F16 gauges (24 B per
 *          site), with or without a U(1) phase field (a 32^4 lattice fits at FP64); larger
 *          lattices return STG_ERR_ARG before any launch.
 *   Arguments: in and out must not overlap (STG_ERR_ARG otherwise: the fused epilogue reads in
 *          while it writes out); both 16-byte aligned.
 *   Set-up: the first call on a device looks up the array's device address (cudaGetSymbolAddress
 *          with that device current) and caches it; make that first call before any stream
 *          capture.  Nothing is allocated, here or later.
 *   Sharing: every call on a device uses the same array, which keeps the last call's contents
 *          (each call overwrites all it reads, so nothing must start at zero); calls that overlap
 *          on the GPU (different streams, no ordering) race on it.
 * pq_dev may be NULL (no reduction). */
stg_status stg_normal_op_noalloc(const stg_gauge *g, double mass, double shift, void *out_even_dev,
                                 const void *in_even_dev, double *pq_dev, void *stream);

/* ---- multi-shift CG (Sec. 2, Eq. shift_eo) ------------------------------------------------- */

typedef struct {
    int32_t nshift;          /* 1 .. 32 poles                                                     */
    const double *shifts;    /* host [nshift], sigma_i >= 0                                        */
    double mass;             /* m                                                                 */
    double tol;              /* target relative FP64 true residual |b - A_i x_i| / |b| per shift   */
    int32_t max_iter;        /* iteration cap of each phase (> 0)                                 */
    double inner_tol;        /* mixed solves: stopping residual of the inner multi-shift phase
                                (0 -> 1e-8 for F32 gauges, 1e-4 for BF16/F16 gauges)             */
    double reliable_delta;   /* mixed solves: reliable update once |r| fell by this factor since
                                the last one (0 -> 1e-3)                                          */
    int32_t log_rows;        /* optional: rows of scalar_log to fill (0 = none)                    */
    double *scalar_log;      /* host [log_rows][2 + nshift]: alpha_k, beta_k, zeta_i^{k+1} of the
                                first multi-shift iterations of system 0                         */
    int32_t history;         /* mixed solves, multi-shift phase: residuals kept per window of the
                                deferred solution update (x_i, p_i of every shift formed once per
                                window from the stored FP32 residuals instead of every
                                iteration); 0 -> automatic (up to 256 within 16 GiB of residual
                                storage per solve), 1 -> per-iteration updates, >= 2 -> that many
                                (rounded down to a multiple of 8, at least 8, at most 256);
                                < 0 -> STG_ERR_ARG                                               */
} stg_mscg_params;

typedef struct {
    int32_t iters;            /* multi-shift iterations                                            */
    int32_t reliable_updates; /* FP64 true-residual recomputations during refinement               */
    int32_t refine_iters;     /* largest refinement iteration count over the shifts                */
    double *true_resid;       /* host [nshift] (may be NULL): final |b - A_i x_i| / |b|.  Pure FP64
                                 solves: the FP64 residual.  Mixed solves whose tol is at least
                                 ten times e_i = 64 * 2^-44 (1 + 16 / (m^2 + sigma_i)) for every
                                 shift: the double-single residual (FP64-verified for shifts it
                                 does not clear by e_i).  Tighter mixed solves: the FP64 residual of
                                 the multi-shift solution, updated by - A y in double-single for
                                 every refinement correction y                                   */
    int32_t *shift_iters;     /* host [nshift] (may be NULL): multi-shift iteration at which each
                                 shift stopped                                                    */
    double *inner_resid;      /* host [nshift] (may be NULL): true residual of each shift right
                                 after the multi-shift phase, before refinement                   */
    int32_t fp64_fallback;    /* 1 if a mixed solve was repeated with FP64 reliable updates       */
    int32_t *refine_shift_iters;  /* host [nshift] (may be NULL): refinement CG iterations of each
                                     shift (0 for shifts the multi-shift phase finished)          */
    int32_t *shift_reliable_updates; /* host [nshift] (may be NULL): reliable updates of each shift's
                                     refinement                                                   */
} stg_mscg_stats;

/* Solves A_{sigma_i} x_i = b for every shift.
 *   g_f64    F64 gauge (RECON18 or RECON12): true residuals, reliable updates, refinement.
 *   g_inner  NULL -> pure FP64 solve.  Otherwise an F32/BF16/F16 gauge on the same lattice:
 *            multi-shift phase in that precision (FP32 vectors, FP64 scalars and reductions,
 *            solutions accumulated in double-single), then each shift above tol is refined by CG
 *            (FP32 links) with reliable updates in double-single arithmetic.  When tol is loose
 *            enough for double-single residuals to certify every shift, the residuals are
 *            recomputed in double-single and any the bound does not clear is checked in FP64 (the
 *            solve is repeated with FP64 reliable updates if one fails); otherwise the residual of
 *            each multi-shift solution is computed once in FP64 and each reliable update
 *            subtracts A y of its correction y in double-single (see true_resid).
 *   b_c128_dev          canonical complex128 [Vh][3] even-site source (device).
 *   x_c128_dev[nshift]  canonical complex128 [Vh][3] outputs (device), may not alias b.
 * Synchronises `stream` before returning.  STG_ERR_NOCONV if a shift is still above tol
 * after max_iter (stats filled, x holds the last iterate). */
stg_status stg_mscg_solve(const stg_gauge *g_f64, const stg_gauge *g_inner, const stg_mscg_params *params,
                          const void *b_c128_dev, void *const *x_c128_dev, stg_mscg_stats *stats, void *stream);

/* A rational function of the shifted normal operator applied to a field (Sec. 2: the RHMC's
 * rational approximation of a fractional power, one pole per system of Eq. shift_eo):
 *   out = alpha0 b + sum_i residues[i] (m^2 + sigma_i - D_eo D_oe)^-1 b,   sigma_i = params->shifts[i]
 * the systems solved by stg_mscg_solve with params (and g_inner as there), the terms added in pole
 * order in FP64.  The pseudofermion heatbath (power +1/8 per rooted staggered flavour) and the
 * fermion action (power -1/4) are both of this form.  b, out: canonical complex128 even fields
 * (device, may alias); stats as for stg_mscg_solve (may be NULL).  Allocates nshift FP64 fields
 * from the stream-ordered allocator; synchronises like stg_mscg_solve. */
stg_status stg_rational_apply(const stg_gauge *g_f64, const stg_gauge *g_inner, const stg_mscg_params *params,
                              double alpha0, const double *residues, const void *b_c128_dev, void *out_c128_dev,
                              stg_mscg_stats *stats, void *stream);

/* The fermion action of one pseudofermion b from the solutions of its shifted systems (Sec. 2:
 * the RHMC writes the fractional power of the staggered operator as a rational function, a
 * constant plus one pole per system of Eq. shift_eo, and the action as b^dag R(A) b):
 *   S = alpha0 |b|^2 + sum_i residues[i] Re(b^dag x_i),   x_i = (m^2 + sigma_i - D_eo D_oe)^-1 b
 *   lat                  the lattice of the fields
 *   nshift               0 .. 32 (0: alpha0 |b|^2 alone)
 *   residues             host [nshift]
 *   b_c128_dev           canonical complex128 [Vh][3] even-site field (device, 16-byte aligned)
 *   x_c128_dev[nshift]   host array of device pointers to the solutions, same layout (for
 *                        example the outputs of stg_mscg_solve)
 *   s_dev                one device double (8-byte aligned) receiving S
 * The sum runs in FP64 in a fixed order (per element in pole order, fixed block trees over a fixed
 * grid, then one fixed-order sum of the 1024 block partials), so S does not depend on timing.
 * Asynchronous on `stream`; takes an 8 KiB workspace from the stream-ordered allocator.
 * STG_ERR_ARG on a null or misaligned pointer or nshift outside 0..32. */
stg_status stg_pseudofermion_action(const stg_lattice *lat, int32_t nshift, double alpha0, const double *residues,
                                    const void *b_c128_dev, const void *const *x_c128_dev, double *s_dev,
                                    void *stream);

/* One lattice of a batched solve: nrhs sources (pseudofermions) on the same gauge. */
typedef struct {
    const stg_gauge *g_f64;
    const stg_gauge *g_inner;  /* all instances of a batch are mixed, or none is                  */
    int32_t nrhs;              /* 1 .. 16                                                          */
    const void *const *b;      /* [nrhs] canonical complex128 sources (device)                     */
    void *const *x;            /* [nrhs * nshift] outputs, x[r * nshift + i] (device)              */
    stg_mscg_stats *stats;     /* [nrhs] (may be NULL)                                             */
} stg_instance;

/* Solves every (instance, rhs, shift) system of a batch of lattices of different sizes
 * together: each iteration launches one set of kernels for the whole batch, link loads are
 * shared by the rhs of an instance, converged systems are masked out.  Shifts, mass, tol
 * from params (shared).  1 <= ninst <= 16. */
stg_status stg_mscg_solve_batched(int32_t ninst, const stg_instance *inst, const stg_mscg_params *params,
                                  void *stream);

/* ---- fermion force ------------------------------------------------------------------------------ */

/* For S = sum_i r_i Re(b^dag x_i) with x_i = A_{sigma_i}^{-1} b (the solutions passed in),
 * computes per link (z, mu), with y_i = D_oe x_i and u = u_mu(z):
 *   W = + sum_i r_i u y_i(z+mu) x_i(z)^dag   (z even)
 *   W = - sum_i r_i u x_i(z+mu) y_i(z)^dag   (z odd)
 * so that dS = Re tr(dU W) under a change dU of that link, and writes
 *   kind 0: F = TA(U W) = (Z - Z^dag)/2 - tr(Z - Z^dag)/6,  Z = U W   (dS/deps = tr(X F) along
 *           U -> exp(eps X) U, X in su(3)), or
 *   kind 1: W^dag = dS/dRe U + i dS/dIm U.
 * y_i is computed with a double-single (FP32-pair, 48-bit significand) copy of the links, which
 * the F64 gauge creates on first use and keeps; W and F are accumulated in FP64.
 * x_c128_dev[nshift]: canonical complex128 even fields (device);
 * out_c128_dev: canonical complex128 [4][V][3][3] (device).  g_f64 must be an F64 gauge. */
stg_status stg_fermion_force(const stg_gauge *g_f64, int32_t nshift, const double *residues,
                             const void *const *x_c128_dev, void *out_c128_dev, int32_t kind, void *stream);
/* stg_fermion_force at a chosen precision.  prec = STG_F64: exactly stg_fermion_force (out
 * complex128).  prec = STG_F32 (single-precision MD forces, Sec. 5.4): x_i rounded to FP32, y_i from
 * the FP32 12-real companion of the links (created on first use and kept, like the double-single
 * one), W and the output in FP32 arithmetic; out_dev is canonical complex64 [4][V][3][3].  Relative
 * accuracy ~1e-6 against the F64 force.  STG_ERR_ARG for any other prec. */
stg_status stg_fermion_force_prec(const stg_gauge *g_f64, stg_prec prec, int32_t nshift, const double *residues,
                                  const void *const *x_c128_dev, void *out_dev, int32_t kind, void *stream);

/* ---- stout smearing ----------------------------------------------------------------------------- */

/* k-times stout-smeared links U^(k) from U^(0) (the Dirac operator's links, Sec. 2; the smearing
 * step is Morningstar and Peardon's).  One step, per link (x, mu), all links in parallel:
 *   C = rho sum_{nu != mu} [U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)]
 *   i Q = TA(C U^dag),   U' = exp(i Q) U
 * with periodic links in all four directions.  exp(i Q) = f0 + f1 Q + f2 Q^2, the f_j summed
 * from the Taylor series of exp reduced by the Cayley-Hamilton identity Q^3 = c1 Q + c0
 * (c0 = det Q, c1 = tr Q^2 / 2) to the precision's accuracy.
 * prec STG_F64: complex128 arrays, FP64 arithmetic; STG_F32: complex64 arrays, FP32 arithmetic
 * (the molecular dynamics runs in single precision, Sec. 5.4).
 * links_dev: canonical [4][V][3][3] U^(0) (device, read only);
 * levels_dev: nstep consecutive canonical arrays U^(1) .. U^(nstep) (device, written).
 * 1 <= nstep <= 16, |rho| <= 0.5 (larger rho is refused: the series would cancel digits);
 * no aliasing between the two buffers; both 16-byte aligned.  Async on `stream`. */
stg_status stg_stout_smear(const stg_lattice *lat, stg_prec prec, int32_t nstep, double rho, const void *links_dev,
                           void *levels_dev, void *stream);

/* Force chain rule through the smearing (Sec. 3: the MD evolves U^(0) while the fermion action
 * depends on U^(k)).  Given G_k = dS/dRe U^(k) + i dS/dIm U^(k) (e.g. stg_fermion_force kind 1
 * evaluated on U^(k)), pulls it back one step at a time, per link, with G' the gradient of U':
 *   M = G' U^dag,  G_Q = K1 Q + K0 Q^2 + conj(f1) M + conj(f2) (M Q + Q M),
 *   K1 = sum_j Re(tr(M^dag Q^j) df_j/dc1),  K0 = sum_j Re(tr(M^dag Q^j) df_j/dc0),
 *   G_Omega = TA(i G_Q),  G = exp(iQ)^dag G' + G_Omega^dag C + (staple terms of rho G_Omega U)
 * where the staple terms collect, for every link, the product-rule terms of the six staples of
 * the three other directions that contain it (a gather: no atomics, deterministic).
 * links_dev: U^(0); levels_dev: the stg_stout_smear output (U^(1) .. U^(nstep-1) are read);
 * grad_dev: G_k; out_dev: kind 1: G_0 = dS/dRe U^(0) + i dS/dIm U^(0), kind 0:
 * F = TA(U^(0) G_0^dag) (dS/deps = tr(X F) along U^(0) -> exp(eps X) U^(0)).
 * All canonical [4][V][3][3] device arrays of prec (F64: complex128, F32: complex64); out must not
 * alias the inputs.  Allocates 2 link-sized work arrays from the stream-ordered allocator.  Same
 * limits as smearing. */
stg_status stg_stout_force(const stg_lattice *lat, stg_prec prec, int32_t nstep, double rho, const void *links_dev,
                           const void *levels_dev, const void *grad_dev, void *out_dev, int32_t kind, void *stream);

/* ---- gauge action and force --------------------------------------------------------------------- */

/* Tree-level Symanzik gauge action of the unsmeared links (Sec. 2; its force is the gauge term of the
 * MD force, Sec. 3), links periodic in all four directions:
 *   S_g = -(beta/3) sum_x sum_{mu != nu} [ 5/6 Re tr P_{mu nu}(x) - 1/12 Re tr R_{mu nu}(x) ]
 *   P_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag                     (1x1 plaquette)
 *   R_{mu nu}(x) = U_mu(x) U_mu(x+mu) U_nu(x+2mu) U_mu(x+mu+nu)^dag U_mu(x+nu)^dag U_nu(x)^dag  (2x1)
 * out3_dev (device, 3 doubles, written): S_g, the plaquette sum sum_{x, mu<nu} Re tr P (each
 * plaquette once) and the rectangle sum sum_{x, mu!=nu} Re tr R (each rectangle once).  The block
 * partial sums are added in a fixed order (bitwise reproducible).  FP64.  Allocates
 * 16 bytes per 128 sites from the stream-ordered allocator; async on `stream`. */
stg_status stg_gauge_action(const stg_lattice *lat, double beta, const void *links_c128_dev, double *out3_dev,
                            void *stream);

/* Gradient of S_g per link: G = dS_g/dRe U + i dS_g/dIm U = -(beta/3) sum c B^dag over the loops
 * through the link (B = the rest of the loop after the link; 2 plaquettes and 6 rectangles per
 * other direction), written as kind 1: G, or kind 0: F = TA(U G^dag) (dS/deps = tr(X F) along
 * U -> exp(eps X) U).  prec STG_F64: complex128 arrays, FP64; STG_F32: complex64 arrays, FP32 (the
 * single-precision MD, Sec. 5.4).  links_dev / out_dev: canonical [4][V][3][3] (device), no
 * aliasing.  Async on `stream`. */
stg_status stg_gauge_force(const stg_lattice *lat, stg_prec prec, double beta, const void *links_dev, void *out_dev,
                           int32_t kind, void *stream);

/* ---- molecular dynamics (Sec. 2-3) ----------------------------------------------------------------- */
/* The MD evolves links U and momenta H (traceless Hermitian, one per link) under
 * (1/2) sum tr H^2 + S(U):  U' = i H U,  H' = -i F  with F = TA(U G^dag) the Lie-algebra force of S
 * (stg_gauge_force / stg_stout_force / stg_fermion_force kind 0 format).  All arrays canonical
 * complex128 [4][V][3][3] (device, 16-byte aligned); FP64; async on `stream`. */

/* Momentum heatbath from caller-drawn standard normal numbers xi_dev [4][V][8] (FP64, device):
 * H = sum_a xi_a lambda_a / sqrt(2) (Gell-Mann matrices), so (1/2) tr H^2 = (1/2) sum_a xi_a^2. */
stg_status stg_md_momenta(const stg_lattice *lat, const double *xi_dev, void *mom_c128_dev, void *stream);
/* U <- exp(i eps H) U for every link (exp by the Cayley-Hamilton series, as in stg_stout_smear);
 * |eps| <= 1; momenta and links must not alias. */
stg_status stg_md_update_links(const stg_lattice *lat, double eps, const void *mom_c128_dev, void *links_c128_dev,
                               void *stream);
/* H <- H - eps i F for every link; the force F in complex128 (force_prec STG_F64) or complex64
 * (STG_F32: a force computed in single precision), the momenta complex128. */
stg_status stg_md_update_momenta(const stg_lattice *lat, stg_prec force_prec, double eps, const void *force_dev,
                                 void *mom_c128_dev, void *stream);
/* dst[k] = src[k] for `count` complex numbers, converting between complex128 (STG_F64) and
 * complex64 (STG_F32) (device arrays, 16-byte aligned, no aliasing): the links and forces of the
 * single-precision MD kernels. */
stg_status stg_complex_convert(int64_t count, stg_prec src_prec, const void *src_dev, stg_prec dst_prec, void *dst_dev,
                               void *stream);
/* *out_dev (one device double) = (1/2) sum_links tr H^2, summed in a fixed order. */
stg_status stg_md_kinetic(const stg_lattice *lat, const void *mom_c128_dev, double *out_dev, void *stream);

/* ---- one-dimensional slab decomposition along t (Sec. 3.1, Sec. 4.1, Sec. 4.2, Alg. 1) ----------
 * The paper tiles the lattice along one direction only: every process holds whole x-y-z volumes of a
 * range of time slices, so that the data it exchanges with its two neighbours are contiguous time
 * slices (no gather or scatter), and D needs one halo slice of the input field on each side.  Here a
 * process (one GPU) holds global slices [t0, t0 + Lt_loc) of a Lx x Ly x Lz x Lt_global lattice.  Its
 * fields and links are stored over Lt_loc + 4 time slices in the usual layouts: the local slices at
 * stored slices 2 .. Lt_loc + 1, the lower neighbour's last slice at stored slice 1, the upper
 * neighbour's first slice at stored slice Lt_loc + 2 (the halos), and stored slices 0 and Lt_loc + 3
 * as padding that keeps the stored parity equal to the global one.  The caller moves the halos
 * (stg_slab_layout gives the byte ranges; the Python binding does it over torch.distributed); the
 * library computes.  No device code waits on another process. */

/* A slab lattice.  dims_local = {Lx, Ly, Lz, Lt_loc}, all even and >= 2; t0 even, Lt_global even,
 * t0 + Lt_loc <= Lt_global.  The antiperiodic sign sits on the t-links at global time
 * Lt_global - 1.  stg_lattice_sites and stg_field_bytes count stored sites (halos included);
 * stg_field_pack / unpack and stg_gauge_create / update take stored canonical arrays (the links of
 * stored slice 1 must hold the lower neighbour's, of which D reads the t-links).  On a slab,
 * stg_dslash / _eo / _oe / _multi and the stg_slab_* calls write the local slices only and read the
 * input's halo slices; every other entry point returns STG_ERR_SHAPE. */
stg_status stg_lattice_create_slab(const int32_t dims_local[4], int32_t t0, int32_t Lt_global, int32_t t_antiperiodic,
                                   stg_lattice **out);
/* Byte layout of a slab field of vector precision vec_prec (F64, DS or F32), for the halo exchange:
 * the internal field is *nchunk arrays, array k starting at byte offset[k] of the field with
 * elem_bytes[k] bytes per site, and stored time slice s of the parity occupying sites
 * [s * slice_sites, (s + 1) * slice_sites) of every array (time is the slowest coordinate), i.e.
 * bytes offset[k] + elem_bytes[k] * [s * slice_sites, (s + 1) * slice_sites).  Exchange: stored slice
 * 2 goes to the lower neighbour's stored slice Lt_loc + 2, stored slice Lt_loc + 1 to the upper
 * neighbour's stored slice 1 (neighbours wrap around: the time direction is closed).  Host only. */
stg_status stg_slab_layout(const stg_lattice *lat, stg_prec vec_prec, int32_t *nchunk, int64_t offset[3],
                           int32_t elem_bytes[3], int64_t *slice_sites);

/* D (D_eo for out_parity 0, D_oe for 1) on part of a slab's local slices, the split of Alg. 1:
 * part 1 the two border slices (stored slices 2 and Lt_loc + 1, in one launch), part 2 the bulk
 * (stored slices 3 .. Lt_loc; nothing when Lt_loc = 2), part 0 every local slice (as stg_dslash).
 * The border outputs can then travel to the neighbours while the bulk computes on another stream
 * (the bulk writes none of the bytes the exchange reads or writes).  in's halo slices must be
 * current.  STG_ERR_ARG for another part; STG_ERR_SHAPE on a full lattice. */
stg_status stg_slab_dslash_part(const stg_gauge *g, int32_t out_parity, int32_t part, void *out_dev, const void *in_dev,
                                void *stream);
/* out = coef p - D in on the output sites (the local slices of a slab, every site of a full
 * lattice): D_eo for out_parity 0, D_oe for 1 (the second half of Eq. shift_eo's operator, with
 * coef = m^2 + sigma).  pq_dev != NULL receives this process's part of Re<p, out> (FP64, fixed
 * order).  Fields in the gauge's internal layout; in's halo slices must be current.  Uses the
 * gauge's partial-sum buffer (concurrent calls on one gauge race, as for stg_normal_op). */
stg_status stg_slab_dslash_xpay(const stg_gauge *g, int32_t out_parity, double coef, void *out_dev, const void *in_dev,
                                const void *p_dev, double *pq_dev, void *stream);
/* y += alpha x on the output sites (the local slices of a slab), fields of vector precision
 * vec_prec F64 or F32 in the internal layout of lat; norm2_dev != NULL receives this process's
 * part of |y|^2 after the update (FP64, fixed order).  Takes a workspace of one double per 256
 * sites from the stream-ordered allocator. */
stg_status stg_slab_axpy_norm(const stg_lattice *lat, stg_prec vec_prec, double alpha, const void *x_dev, void *y_dev,
                              double *norm2_dev, void *stream);
/* The multi-shift update of the solutions and search directions (Sec. 2) on the output sites:
 * for i < n, x_i += cx[i] p_i if upd_x[i], then p_i = cr[i] r + cp[i] p_i if upd_p[i]; host arrays
 * of n <= 32 coefficients and flags, device pointers x[i], p[i], r in the internal layout
 * (vec_prec F64 or F32). */
stg_status stg_slab_shift_update(const stg_lattice *lat, stg_prec vec_prec, int32_t n, const double *cx,
                                 const double *cr, const double *cp, const int32_t *upd_x, const int32_t *upd_p,
                                 void *const *x_dev, void *const *p_dev, const void *r_dev, void *stream);

/* Host-side scalar recurrences of the multi-shift CG (Sec. 2, Eq. shift_eo; the shifted CG of
 * Jegerlehner) for a driver that sums its reductions over processes itself: base shift
 * sigma_0 = min sigma_i, relative shifts s_i = sigma_i - sigma_0, and per iteration
 *   stg_mscg_state_alpha with Re<p, q> (summed over processes):  alpha = |r|^2 / Re<p, q>,
 *     zeta_i' = zeta_i zeta_i_old alpha_old / (alpha beta_old (zeta_i_old - zeta_i)
 *                                              + zeta_i_old alpha_old (1 + s_i alpha)),
 *     cx_i = alpha zeta_i' / zeta_i  (x_i += cx_i p_i);
 *   stg_mscg_state_beta with |r|^2 after r -= alpha q:  beta = |r|^2_new / |r|^2,
 *     cr_i = zeta_i', cp_i = beta (zeta_i' / zeta_i)^2  (p_i = cr_i r + cp_i p_i), the stop test
 *     zeta_i' |r| <= tol |b| per shift, the base direction kept while any shift runs, and the
 *     history rotation; state.running = 0 once every shift has stopped or max_iter is reached.
 * Plain FP64 host arithmetic, no GPU needed.  STG_ERR_ARG on a NULL state, nshift outside 1..32,
 * a negative shift, or a step called out of order. */
typedef struct {
    int32_t nshift, i0, iters, max_iter, running, nactive, phase;  /* phase 0: alpha next, 1: beta next */
    double s[32], zeta[32], zeta_old[32], zeta_new[32];
    double alpha, alpha_old, beta_old, rr, tol2;
    double cx[32], cr[32], cp[32];
    int32_t active[32], upd_x[32], upd_p[32], shift_iters[32];
} stg_mscg_state;
stg_status stg_mscg_state_init(stg_mscg_state *st, int32_t nshift, const double *shifts, double tol, double bnorm2,
                               int32_t max_iter);
stg_status stg_mscg_state_alpha(stg_mscg_state *st, double pq);
stg_status stg_mscg_state_beta(stg_mscg_state *st, double rr_new);

#ifdef __cplusplus
}
#endif
#endif /* STG_H */
