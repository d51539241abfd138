/*
 * vie.h - C ABI of libvie: the FFT-based volume-integral-equation (VIE)
 * operator whose circulant Green's-function tensors are held Tucker
 * (HOSVD) compressed, its adjoint, and the GMRES solve built on it.
 *
 * Method: Giannakopoulos, Litsarev, Polimeridis, "Memory footprint reduction
 * for the FFT-based volume integral equation method via tensor
 * decompositions".  Problem statement: the J-block of eqs. (1)-(4),
 *     (M_eps_r - M_chi N) j = c_e M_chi e_inc ,
 * with N of eq. (5) and the Green's function g of eq. (6).  Writing
 * N = G + I, where G = (k0^2 + grad div) applied to the vector potential,
 * and w = j / c_e, this is the library's system
 *     A w = w - chi * (G w) = chi * e_inc .                        (S)
 *
 * Discretisation (uniform n1 x n2 x n3 grid of voxels of edge h, Section
 * II.B): G is block-Toeplitz with Toeplitz blocks; its six unique dyadic
 * components T_ab (ab = xx, xy, xz, yy, yz, zz) are the kernel
 * (k0^2 delta_ab + d_a d_b) g sampled at voxel-centre offsets times h^3, and
 * at zero offset the field of a uniform unit source in the equivalent
 * sphere of radius a = h (3/4pi)^(1/3):
 *     T_ab(0) = delta_ab [ (2/3)(1 + i k0 a) exp(-i k0 a) - 1 ].
 * Each component is embedded in a circulant tensor of size
 * P1 x P2 x P3 (P_q = 2 n_q; wrap-around planes at index n_q hold zero),
 * DFT'd (Section V.A) and compressed by truncated HOSVD (Algorithm 1) to a
 * core of size r1 x r2 x r3 and factors U^q (P_q x r_q), eqs. (13)-(14).
 * The matvec (Section V.B) zero-pads and 3-D FFTs the current, rebuilds the
 * components from core and factors (or, after vie_tucker_cp, from the
 * Tucker+CP factors of Algorithm 2, eq. (17)), multiplies voxel by voxel,
 * inverse-FFTs and crops.
 *
 * Conventions for every call:
 *  - Arrays are C order, z fastest.  Vector fields are [B][3][n1][n2][n3]
 *    (component a = x, y, z), scalar fields [n1][n2][n3].
 *  - Complex numbers are interleaved (re, im): "c64" = 2 x float,
 *    "c128" = 2 x double.  `precision` selects VIE_C64 or VIE_C128 for the
 *    array arguments of a call.
 *  - Pointers marked "device" must be CUDA device (or managed) memory owned
 *    by the caller; the library never frees them.  Pointers marked "host"
 *    are ordinary host memory.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    asynchronous on it unless stated otherwise.
 *  - Every call returns a vie_status; a non-zero status leaves outputs
 *    unspecified and is never signalled by abort().  vie_last_error()
 *    returns a message for the last failure on the calling thread.
 *  - Scratch memory is owned by the vie_op and grows on demand; call
 *    vie_reserve() first if later calls must not allocate (for example
 *    inside CUDA graph capture).
 */
#ifndef VIE_H
#define VIE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum vie_status {
    VIE_OK = 0,
    VIE_ERR_ARG = 1,             /* invalid argument or unsupported size      */
    VIE_ERR_CUDA = 2,            /* a CUDA runtime call or launch failed      */
    VIE_ERR_OOM = 3,             /* device or host allocation failed          */
    VIE_ERR_NO_CONVERGENCE = 4,  /* solver hit its iteration limits           */
    VIE_ERR_NUMERIC = 5,         /* NaN/Inf, breakdown or eigen-solver failure */
    VIE_ERR_TIMEOUT = 6          /* a bounded device wait ran out             */
} vie_status;

enum { VIE_C64 = 0, VIE_C128 = 1 };                 /* array precision          */
enum { VIE_PATH_TUCKER = 0, VIE_PATH_UNCOMPRESSED = 1,
       VIE_PATH_TUCKER_CP = 2 };            /* after vie_tucker_cp; FP32 only */

/* HOSVD truncation rule (Algorithm 1; the printed rule is garbled):
 * TAIL      - smallest r_q with sqrt(sum_{j>r_q} sigma_j^2) <= (tol/sqrt3)||A||_F,
 *             which bounds ||A - A~||_F <= tol ||A||_F (eq. (12));
 * SIGMA_MAX - keep sigma_j >= (tol/sqrt3) sigma_max.                           */
enum { VIE_RANK_TAIL = 0, VIE_RANK_SIGMA_MAX = 1 };

/* vie_tucker_compress flags */
enum {
    VIE_STORE_UNCOMPRESSED = 1,  /* also keep the six full spectra (the paper's
                                    "traditional FFT-JVIE", Table II row 1) in
                                    c64 and c128, for VIE_PATH_UNCOMPRESSED     */
    VIE_SELF_TERM_PV = 2,        /* self term without the -1/3 depolarisation  */
    VIE_REBUILD_SIMT = 4,        /* rebuild the half fibres of eq. (13) with
                                    FP32 CUDA-core FMAs instead of the tensor
                                    cores (3xTF32 mma); for comparison          */
    VIE_REBUILD_TCGEN05 = 16,    /* rebuild on the tensor cores through
                                    tcgen05.mma with the accumulator in tensor
                                    memory instead of warp-level mma.sync
                                    (both 3xTF32); for comparison: slower on
                                    the rebuild's small K (2 r3)              */
    VIE_SETUP_FACTORWISE = 8     /* Section V.A: compress the Toeplitz defining
                                    tensor (its parity octant, n1 n2 n3) and
                                    embed + DFT the factor columns, instead of
                                    compressing the FFT'd P1 P2 P3 circulant
                                    tensor; the same ranks and model, without
                                    forming the P1 P2 P3 spectrum (unless the
                                    spectra are stored)                          */
};

/* vie_solve flags */
enum {
    VIE_SOLVE_ADJOINT = 1,       /* solve A^H w = b instead of A w = b          */
    VIE_SOLVE_RHS_INCIDENT = 2,  /* `rhs` is e_inc and b = chi * e_inc; else
                                    `rhs` is b itself                           */
    VIE_SOLVE_X0 = 4             /* `w` holds the initial guess on entry        */
};

typedef struct vie_grid {
    int n1, n2, n3;      /* voxels per axis (x, y, z), each >= 1             */
    double h;            /* voxel edge, metres (> 0)                          */
    double freq_hz;      /* frequency; k0 = 2 pi f / c with c = 299792458 m/s */
} vie_grid;

typedef struct vie_op vie_op;    /* opaque; owns the device core/factors */

typedef struct vie_op_info_t {
    int n[3];                    /* grid                                       */
    int P[3];                    /* padded (circulant) sizes 2 n_q              */
    int ranks[6][3];             /* multilinear ranks per component (xx..zz)   */
    size_t tucker_bytes;         /* c64 cores + factors as stored (half rows)   */
    size_t tucker_bytes_full;    /* c64 cores + full factors (P_q rows), eq. (13)*/
    size_t slab_bytes;           /* c64 slab cores core x1 U1[k1,:] for the
                                    P1/2+1 rows k1 (formed at setup, reused by
                                    every matvec)                               */
    size_t rebuild_scratch_bytes;/* c64 scratch into which every Tucker matvec
                                    rebuilds the half fibres of a chunk of k1
                                    (at most 64 MiB; 0 when the grid takes the
                                    shared-memory path, which rebuilds on chip) */
    size_t uncompressed_bytes;   /* six c64 spectra, 6 P1 P2 P3 x 8 bytes       */
    size_t workspace_bytes;      /* scratch currently held                      */
    int has_uncompressed;        /* VIE_STORE_UNCOMPRESSED was given            */
    int max_batch;               /* c64 batch size the matvec scratch serves
                                    (half of it in c128)                        */
    int line_threads[4];         /* CTA size of the x, y, inverse y, inverse x
                                    FFT stages (vie_autotune's choice)          */
    int tuned_batch;             /* batch vie_autotune timed at (0 = defaults)  */
    int rebuild_kernel;          /* how each FP32 Tucker matvec rebuilds the
                                    half fibres: 0 inside the fused z-stage
                                    CTAs (no scratch), 1 FP32 FMAs into the
                                    scratch, 2 tensor cores through warp-level
                                    mma.sync (3xTF32) into it, 3 tensor cores
                                    through tcgen05.mma with TMEM accumulators
                                    (3xTF32) into it                          */
    int cp_rank;                 /* terms R of the Tucker+CP model (0: none)   */
    double cp_rel_err[6];        /* ||core - CP|| / ||core|| per component;
                                    the factors U^q are orthonormal, so this
                                    is also the Tucker+CP error relative to
                                    the Tucker model                           */
    int cp_sweeps[6];            /* ALS sweeps taken per component             */
    size_t cp_bytes;             /* c64 Tucker+CP factors W^q (half rows)      */
    size_t device_bytes_tucker;  /* all device memory the operator holds for the
                                    compressed paths: c64 and c128 cores and
                                    half factors, slab cores, the rebuild's U3
                                    fragments and scratch, Tucker+CP factors,
                                    metadata and FFT root tables               */
    size_t device_bytes_spectra; /* stored spectra, c64 and c128 (0 without
                                    VIE_STORE_UNCOMPRESSED)                     */
    size_t matvec_workspace_bytes; /* matvec scratch T1 + T2 currently held     */
    size_t solver_workspace_bytes; /* Krylov basis, Hessenberg, refinement
                                    vectors currently held (vie_solve)         */
    size_t setup_scratch_bytes;  /* device scratch vie_tucker_compress held while
                                    compressing (released before it returned):
                                    the FP64 P1 P2 P3 spectrum of one component
                                    (spectrum route, or stored spectra), the
                                    weighted octant, Gram matrices and vectors  */
    int rebuild_tiles[2];        /* rebuild_kernel 3: k3 columns of a CTA's
                                    range and CTAs per (component, range)
                                    (vie_autotune's choice, else the default
                                    of one CTA per SM); 0 otherwise            */
} vie_op_info_t;

/* vie_solve options (Section VI.C: GMRES, inner 50 / outer 200). */
typedef struct vie_solve_opts {
    double tol;          /* target FP64 relative residual ||b - A w||/||b||   */
    int restart;         /* GMRES restart length m (1..128)                    */
    int max_outer;       /* restart cycles allowed per inner solve            */
    double inner_tol;    /* relative tolerance of each FP32 inner solve       */
    int max_refine;      /* FP64 refinement steps allowed (<= 64)              */
    int path;            /* VIE_PATH_TUCKER or VIE_PATH_UNCOMPRESSED            */
    int use_graph;       /* replay each restart cycle as a CUDA graph         */
    int refine;          /* 1: FP64 iterative refinement; 0: FP32 GMRES only  */
    int orth;            /* Arnoldi: 2 = classical Gram-Schmidt with a second
                            pass when the DGKS test asks (||w'|| < ||w||/sqrt2),
                            1 = one classical pass (the FP64 refinement
                            absorbs the orthogonality loss)                   */
} vie_solve_opts;

typedef struct vie_solve_info {
    int converged;           /* every RHS reached opts.tol                      */
    int refine_steps;        /* FP64 residual evaluations after the first       */
    int iterations;          /* inner Arnoldi iterations (all steps)            */
    int matvecs;             /* operator applications (FP32 + FP64)             */
    double relres;           /* final relative residual, max over RHS           */
    double history[65];      /* relres after each refinement step               */
} vie_solve_info;

/*
 * Build the compressed operator for `grid` (eqs. (5)-(6), Sections II.B and
 * V.A, Algorithm 1): assemble each of the six defining tensors in FP64 on
 * the device, embed it circulantly, 3-D FFT it, and compress it by
 * truncated HOSVD at relative tolerance `tol` (> 0, < 1) with `rank_rule`.
 * Cores and factors are kept in c64 (matvec) and c128 (refinement).
 * Grid edges 2 n_q must factor into primes <= 7 and n_q <= 512.
 * Synchronises `stream`.  On success *out receives a new operator that the
 * caller releases with vie_destroy().
 */
int vie_tucker_compress(const vie_grid* grid, double tol, int rank_rule,
                        int flags, void* stream, vie_op** out);

/* Sizes, ranks and memory of `op` (host struct, filled on success). */
int vie_op_info(const vie_op* op, vie_op_info_t* info);

/*
 * Copy component c (0..5 = xx, xy, xz, yy, yz, zz) of `op` to host buffers
 * in c128: core [r1][r2][r3], factors U1 [P1][r1], U2 [P2][r2], U3 [P3][r3]
 * (all P_q rows, so that eq. (13) rebuilds the full spectrum) and the
 * singular values of the three unfoldings, sigma_q [P_q/2 + 1] each
 * (descending; the unfolding has at most P_q/2 + 1 nonzero ones).  Any
 * pointer may be NULL.  Synchronises `stream`.
 */
int vie_op_export(const vie_op* op, int c, double* core, double* U1, double* U2,
                  double* U3, double* sigma1, double* sigma2, double* sigma3,
                  void* stream);

/*
 * Tucker+CP (Algorithm 2): a CP model with `rank` terms (1..32) of each of
 * the six HOSVD cores of `op`, core ~ sum_l V1[:, l] o V2[:, l] o V3[:, l],
 * fitted by alternating least squares on the device in FP64 (each sweep
 * solves the least-squares problem of V1, V2, V3 in turn with the other two
 * fixed), from a start fixed by `seed`; sweeps stop when the relative core
 * error changes by less than `tol`, or after `max_iter` sweeps.  Then the
 * Tucker+CP factors W^q = U^q V^q (eq. (17)) are formed, and the FP32
 * matvec, adjoint matvec and solve accept VIE_PATH_TUCKER_CP, which rebuilds
 * the half fibres from eq. (17) at every matvec (in a solve, FP64
 * refinement residuals use the Tucker model).  Calling it again replaces the
 * model.  Needs the rebuild scratch (rebuild_kernel != 0 in vie_op_info).
 * Errors: VIE_ERR_ARG (rank, tol, max_iter, a Tucker rank above 64, no
 * scratch), VIE_ERR_NUMERIC (the fit did not stay finite), VIE_ERR_OOM.
 * Synchronises `stream`.
 */
int vie_tucker_cp(vie_op* op, int rank, double tol, int max_iter,
                  unsigned long long seed, void* stream);

/*
 * Tucker+CP factors of component c to host buffers in c128, W1 [P1][R],
 * W2 [P2][R], W3 [P3][R] (all P_q rows, so that eq. (17) rebuilds the full
 * spectrum), the final relative core error and the sweeps taken.  Any
 * pointer may be NULL.  VIE_ERR_ARG without a model.  Synchronises `stream`.
 */
int vie_cp_export(const vie_op* op, int c, double* W1, double* W2, double* W3,
                  double* rel_err, int* sweeps, void* stream);

/*
 * The uncompressed FFT'd circulant component c (Section V.A) for `grid`,
 * c128 [P1][P2][P3] written to device memory `out`.  The first two steps of
 * vie_tucker_compress, exposed for checking.
 */
int vie_green_spectrum(const vie_grid* grid, int c, int flags, void* out,
                       void* stream);

/* Size the scratch of `op` for batches of up to max_batch vectors, in
 * both precisions.  Synchronous. */
int vie_reserve(vie_op* op, int max_batch);

/*
 * Y = G J for B >= 1 vector fields (Section V.B): zero-pad, 3-D FFT, voxel-
 * wise product with the six components, inverse FFT, crop.  The components
 * are rebuilt at every call from the Tucker form (VIE_PATH_TUCKER, eq. (13):
 * the last two mode products, from slab cores core x1 U1[k1,:] formed at
 * setup) or from the Tucker+CP factors (VIE_PATH_TUCKER_CP, eq. (17), c64
 * only, after vie_tucker_cp), or read from the stored spectra
 * (VIE_PATH_UNCOMPRESSED, operators built with VIE_STORE_UNCOMPRESSED).
 * J, Y: device [B][3][n1][n2][n3] in `precision`; Y may alias J.
 * Errors: VIE_ERR_ARG (NULL, B outside [1, 4096], a path the operator
 * cannot serve, VIE_PATH_TUCKER_CP with VIE_C128), VIE_ERR_OOM (scratch),
 * VIE_ERR_CUDA.
 */
int vie_matvec(const vie_op* op, const void* J, void* Y, int B, int path,
               int precision, void* stream);

/*
 * Y = G J like vie_matvec with path VIE_PATH_TUCKER and precision VIE_C64,
 * but without allocating any memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when
 * they need a product, for example serving loops whose device memory is
 * owned by another allocator under a fixed budget, or callbacks that must
 * not trigger the device-wide synchronisation cudaMalloc and cudaFree can
 * cause.
 * Its scratch is one fixed 64 MiB array compiled into the library (every
 * GPU that loads the library holds it until the process exits).  A call
 * needs 24 B (P1 n2 n3 + P1 P2 n3) bytes of it; larger grids or batches
 * are rejected with VIE_ERR_ARG (use vie_matvec).  Nothing in the scratch
 * needs to start at zero: every call overwrites what it reads.
 * The first call on each device looks up the scratch address (with that
 * device current); make that first call before any stream capture.
 * All calls share the one array (and the operator's rebuild scratch), so
 * calls that overlap on the GPU (different streams, or concurrent host
 * threads) race; serialise them.  J, Y: device [B][3][n1][n2][n3] c64.
 */
int vie_matvec_noalloc(const vie_op* op, const void* J, void* Y, int B,
                       void* stream);

/*
 * Y_p = G_p J_p for `count` operators at once, c64, Tucker path: the batched
 * and mixed-size counterpart of vie_matvec (Section V.B for each operator).
 * Grids of different sizes, each with its own batch B[p], go through one
 * persistent cooperative launch (vie_matvec_multi_ex with
 * VIE_MULTI_PERSISTENT): the five stages (x, y, fused z with the rebuild of
 * each mirror group's half fibres inside its CTA, inverse y, inverse x) run
 * in turn, every CTA taking the stage's work items of all operators, with a
 * grid-wide barrier between stages (bounded by one second of the device
 * timer; a barrier that runs out sets the device error word of ops[0] that
 * vie_solve reports as VIE_ERR_TIMEOUT).  VIE_MULTI_STAGED launches one
 * kernel per stage instead.  Both need every padded edge 2 n_q = 32 R with R
 * in {1..6, 8}; otherwise (or for count > 8, in groups of 8) the problems go
 * through the per-operator path.  ops, J, B: host arrays of `count` entries;
 * J[p], Y[p]: device [B[p]][3][n1][n2][n3] of operator p.  Operators must be
 * distinct (each uses its own scratch).
 */
enum { VIE_MULTI_PERSISTENT = 0, VIE_MULTI_STAGED = 1 };
int vie_matvec_multi_ex(const vie_op* const* ops, const void* const* J, void* const* Y,
                        const int* B, int count, int mode, void* stream);
/* vie_matvec_multi_ex with VIE_MULTI_PERSISTENT. */
int vie_matvec_multi(const vie_op* const* ops, const void* const* J,
                     void* const* Y, const int* B, int count, void* stream);

/*
 * Pick the CTA size (64, 128 or 256 threads) of each register-path FFT
 * stage of `op` by timing FP32 Tucker matvecs at batch B on `stream`, and
 * keep the fastest; then, for the tcgen05 rebuild (rebuild_kernel 3), the
 * tile shape of the rebuild of eq. (13) (k3 columns per CTA and CTAs per
 * component), timed over every k1 chunk of one matvec.  vie_op_info reports
 * the choices.  Allocates two temporary batches; synchronises `stream`.
 * Results of later calls do not change, only their speed.  Do not run it
 * while another stream uses `op`.
 */
int vie_autotune(vie_op* op, int B, void* stream);

/* X = G^H Y = conj(G conj(Y)) (G is complex symmetric).  Layout as vie_matvec. */
int vie_matvec_adjoint(const vie_op* op, const void* Y, void* X, int B,
                       int path, int precision, void* stream);

/*
 * out = A w = w - chi * (G w)        (adjoint = 0), or
 * out = A^H w = w - G^H (conj(chi) w) (adjoint = 1),  the operator of (S).
 * chi: device [n1][n2][n3]; w, out: device [B][3][n1][n2][n3]; out may not
 * alias w.
 */
int vie_apply_system(const vie_op* op, const void* chi, const void* w, void* out,
                     int B, int adjoint, int path, int precision, void* stream);

/* E = e_inc + G w, the total field of (S).  All device [B][3][n1][n2][n3]. */
int vie_total_field(const vie_op* op, const void* einc, const void* w, void* E,
                    int B, int path, int precision, void* stream);

/*
 * Solve (S) or its adjoint for B right-hand sides with GMRES (Section VI.C)
 * in FP32 (c64 Krylov vectors, FP64 dot products, Hessenberg and Givens
 * rotations), wrapped in FP64 iterative refinement when opts->refine:
 * r = b - A w is formed with the FP64 operator and corrected by inner FP32
 * solves until ||r||/||b|| <= opts->tol for every RHS.
 * chi: device [n1][n2][n3]; rhs: device [B][3][n1][n2][n3] (e_inc or b per
 * `flags`); w: device, same layout, receives the solution (and holds x0
 * with VIE_SOLVE_X0).  Synchronises `stream` once per restart cycle.
 * With opts->path = VIE_PATH_TUCKER_CP the inner FP32 solves apply the
 * Tucker+CP model (eq. (17)) and the FP64 residuals the Tucker model it
 * approximates, so the solution is that of the Tucker operator; the
 * refinement converges only while the CP model is close enough to it.
 * Returns VIE_ERR_NO_CONVERGENCE (with `info` filled) if the limits are hit.
 */
int vie_solve(const vie_op* op, const void* chi, const void* rhs, void* w, int B,
              int flags, int precision, const vie_solve_opts* opts,
              vie_solve_info* info, void* stream);

/*
 * Several independent solves, e.g. the mixed-grid batch of 48^3, 64^3 and 80^3
 * problems with their own right-hand sides (Section VI.C solve for each): the
 * `count` solves run concurrently on the device, each as vie_solve would run
 * it (its own internal stream and restart-cycle graphs, driven by its own host
 * thread), so small grids fill the GPU together.  Results are those of `count`
 * separate vie_solve calls.  ops, chi, rhs, w, B: host arrays of `count`
 * entries, laid out as for vie_solve on the respective operator; the
 * operators must be distinct.  flags, precision and opts apply to every
 * solve; info: `count` records or NULL.  Ordered after the work already on
 * `stream`, and the caller's stream waits for every solve.  Returns VIE_OK
 * when every solve did, else the status of the first failing one (the others
 * still complete).  The paper solves one problem at a time; this entry point
 * has no counterpart there.
 */
int vie_solve_multi(const vie_op* const* ops, const void* const* chi, const void* const* rhs,
                    void* const* w, const int* B, int count, int flags, int precision,
                    const vie_solve_opts* opts, vie_solve_info* info, void* stream);

/*
 * Contrast gradient from a forward field E and an adjoint solution lam:
 *   grad[v] = scale * sum_b sum_a lam[b,a,v] conj(E[b,a,v]).
 * For the misfit L = sum |E - E_target|^2 with A^H lam = G^H (E - E_target)
 * and scale = 2 this is dL/dRe chi + i dL/dIm chi (A dw = dchi E, dE = G dw).
 * lam, E: device [B][3][n1][n2][n3]; grad: device [n1][n2][n3].
 */
int vie_contrast_gradient(const vie_op* op, const void* lam, const void* E,
                          void* grad, int B, double scale, int precision,
                          void* stream);

/*
 * Incident fields of B unit z-directed point dipoles at host points
 * `sources` [B][3] (metres, box centre at the origin, voxel centres at
 * (i + 1/2 - n/2) h): e_a(r) = (k0^2 delta_az + d_a d_z) g(r - r_s).
 * out: device [B][3][n1][n2][n3].  A source at a voxel centre is an error.
 */
int vie_incident_dipole(const vie_op* op, const double* sources, int B, void* out,
                        int precision, void* stream);

/*
 * Benchmark instrumentation (no counterpart in the paper).  Between
 * vie_profile_start(mask) and vie_profile_stop() every launch of the kernel
 * families selected by `mask` (bit f = family f in the order line_x, line_y,
 * fused_tucker, fused_stored, line_iy, line_ix, tucker_rebuild, arnoldi_dots,
 * arnoldi_update, arnoldi_small, fp64_vector, setup, matvec_fp64 (every stage
 * of the FP64 refinement matvecs); ~0u = all) is
 * bracketed by CUDA events on the stream it runs on
 * (inside CUDA graphs as event nodes read after each replay), and kernels
 * add the algorithmic bytes they move for active right-hand sides to a
 * per-family device counter.  vie_profile_stop() synchronises the device
 * and fills up to max_entries host records (*count of them), one per family
 * that ran: name, launches, total milliseconds, total algorithmic bytes.
 * Profiling adds two event records per launch; it is off by default.
 */
typedef struct vie_profile_entry {
    char name[32];
    long long launches;
    double ms;
    double bytes;
} vie_profile_entry;

int vie_profile_start(unsigned mask);
int vie_profile_stop(vie_profile_entry* out, int max_entries, int* count);

/*
 * Self-test of the bounded device waits (no counterpart in the paper).  The
 * TMA-fed kernels wait on shared-memory barriers for their copies with a
 * limit of one second of the device's global timer; a wait that runs out sets
 * a device word that the next vie_solve synchronisation reports as
 * VIE_ERR_TIMEOUT, and the kernel returns.  This call runs that wait alone in
 * one thread: with arrive = 1 the barrier's arrival is made first and the
 * call returns VIE_OK; with arrive = 0 nothing arrives, the wait gives up
 * after `seconds` (0 < seconds <= 10) and the call returns VIE_ERR_TIMEOUT.
 * arrive = 3 and 2 do the same for the grid barrier of the persistent
 * multi-grid matvec, in a cooperative launch of two CTAs: with 3 both arrive
 * (VIE_OK), with 2 the second never does and the first gives up
 * (VIE_ERR_TIMEOUT).  Synchronises `stream`.
 */
int vie_selftest_bounded_wait(int arrive, double seconds, void* stream);

/* Release `op` and everything it owns (NULL is allowed). */
void vie_destroy(vie_op* op);

/* Static description of a status code. */
const char* vie_status_string(int status);

/* Message for the last failing call on this thread ("" if none). */
const char* vie_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* VIE_H */
