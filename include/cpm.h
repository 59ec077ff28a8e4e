/*
 * cpm.h - C ABI of the GB300 constant potential method (CPM) library.
 *
 * The library computes the two parts of the CPM hot path of the ELECTRODE
 * paper (arXiv 2203.15461):
 *
 *   1. once per electrode geometry: the elastance matrix A of Eq. (coulomb),
 *      Sec. II.A (Gaussian electrode charges of Sec. III.B, Ewald real- and
 *      reciprocal-space sums, self terms, and the slab / wire boundary terms of
 *      Eqs. (ew3dc_slab) and (ew3dc_wire), Sec. II.E), its inverse and the
 *      charge-neutral capacitance matrix S of Eq. (S), Sec. II.A;
 *   2. per MD step and electrolyte configuration: the electrolyte potential b
 *      at every electrode site and the electrode charges q = S (v - b) with
 *      v = G psi (Eq. electrode-wise, Sec. II.B).
 *
 * Sign convention: b_i is the electrostatic potential of the electrolyte at
 * site i (the paper's b with the opposite sign), so q = S (v - b).
 * Units: Angstrom, elementary charge e, volt.  A is in V/e, S in e/V.
 *
 * Every entry point returns a cpm_status and never aborts the process.  All
 * device work is issued on the stream given to cpm_create; calls return when
 * the work is enqueued unless stated otherwise.  Errors raised by kernels
 * (a non-positive Cholesky pivot, a non-finite input) are reported by the
 * next call that synchronises (cpm_invert, cpm_sync, cpm_step_host).
 *
 * Array conventions: "device" pointers are CUDA global memory owned by the
 * caller and only read (or written, for outputs) during the call's stream
 * work; "host" pointers are ordinary host memory.  Coordinates are row-major
 * (N x 3) doubles.  Batched vectors are replica-major: element (r, i) of an
 * (m x n) batch is at [r * n + i].
 */
#ifndef CPM_H
#define CPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CPM_OK = 0,
    CPM_E_ARG = 1,        /* invalid argument (null pointer, bad size or enum) */
    CPM_E_OOM = 2,        /* a device allocation failed */
    CPM_E_BUDGET = 3,     /* the request exceeds the context's device-memory budget */
    CPM_E_NOT_SPD = 4,    /* A is not positive definite (a Cholesky pivot <= 0 or not finite) */
    CPM_E_STATE = 5,      /* call out of order (e.g. cpm_update before cpm_invert) */
    CPM_E_CUDA = 6,       /* a CUDA runtime error; see cpm_last_error */
    CPM_E_TIMEOUT = 7,    /* a bounded device wait expired */
    CPM_E_NONFINITE = 8   /* an input or result is NaN or infinite */
} cpm_status;

/* Periodicity and boundary correction (Sec. II.E). */
typedef enum {
    CPM_BC_3D = 0,    /* 3D periodic, tin-foil: no correction */
    CPM_BC_SLAB = 1,  /* x, y periodic; z padded with vacuum; J = 2 pi M_z^2 / V (Eq. ew3dc_slab) */
    CPM_BC_WIRE = 2,  /* z periodic; x, y padded with vacuum; J = pi (M_x^2 + M_y^2) / V (Eq. ew3dc_wire) */
    CPM_BC_EW2D = 3   /* x, y periodic, z not: the exact 2D Ewald sum (EW2D, Sec. II.E) in place of the 3D
                         reciprocal sum, background and dipole term.  box[2] is no period: it fixes the
                         undetermined constant (2 pi / (Lx Ly)) box[2] of the elastance of a 2D-periodic
                         system (A += c e e^T, b += c Q_tot; S and every neutral result do not depend on
                         it) and must exceed the z range of all sites and charges by rcut.  k_prec FP64 or
                         FP32 (not F16X2); not for cpm_bvec_noalloc. */
} cpm_boundary;

/* Arithmetic of a per-step stage. */
typedef enum {
    CPM_PREC_FP64 = 0,  /* IEEE double throughout */
    CPM_PREC_FP32 = 1,  /* single precision products and accumulation, FP64 neutrality and totals */
    CPM_PREC_BF16X3 = 2, /* s_prec only: S and b each split into three bf16 terms, six products per
                           step on the tensor cores (tcgen05), FP32 accumulation, FP64 split sums */
    CPM_PREC_F16X2 = 3  /* k_prec only: as CPM_PREC_FP32, with the two reciprocal-space contractions
                           (structure factor, site potentials) on the tensor cores (tcgen05): operands
                           scaled by powers of two and split into two fp16 terms, three products,
                           FP32 accumulation */
} cpm_precision;

/* Factorisation of A in cpm_invert (Sec. II.A: A is inverted once per electrode geometry). */
typedef enum {
    CPM_CHOL_FP64 = 0,    /* FP64 blocked Cholesky, triangular inverse, A^-1 = L^-T L^-1 */
    CPM_CHOL_FP32_IR = 1  /* FP32 blocked Cholesky; A X = I refined in FP64 (residual against the FP64 A)
                             until the residual stops shrinking; X symmetrised */
} cpm_chol;

/*
 * Reciprocal-space solver of the per-step electrolyte vector b (cpm_params.kspace).  The paper's
 * package offers an Ewald sum and a particle-particle particle-mesh (P3M) solver (Introduction; SI
 * Sec. 1.A-B).  With CPM_KSPACE_P3M the reciprocal part of b is
 *   phi_i = (1/V) sum_x W_i(x) IFFT[G FFT[rho_mesh]](x),   rho_mesh(x) = sum_j Q_j W_j(x),
 * W the order-p cardinal B-spline assignment function per axis (W(s) = M_p(s + p/2), s in mesh
 * spacings), G the optimal influence function for potentials of Hockney and Eastwood with alias
 * sums over m in [-2, 2]^3:
 *   G(k) = sum_m U^2(k_m) R(k_m) / (sum_m U^2(k_m))^2,  k_m = k + 2 pi m / h,
 *   U(k) = prod_d sinc(k_d h_d / 2)^p,  R(k) = 4 pi exp(-k^2 / 4 alpha^2) / k^2,  G(0) = 0.
 * The elastance matrix A is always assembled with the Ewald sum; the background and the boundary
 * term of b are those of the Ewald path.  Not with CPM_BC_EW2D.
 */
typedef enum {
    CPM_KSPACE_EWALD = 0,
    CPM_KSPACE_P3M = 1
} cpm_kspace;

typedef struct {
    double box[3];       /* Ewald cell (Lx, Ly, Lz) in Angstrom, vacuum padding included */
    int32_t boundary;    /* cpm_boundary */
    double alpha;        /* Ewald splitting parameter (1/Angstrom) */
    double rcut;         /* real-space cut-off: pairs with |r| < rcut over all images count */
    double kcut;         /* reciprocal cut-off: k = 2 pi (nx/Lx, ny/Ly, nz/Lz) counts when
                            ((kx*kx + ky*ky) + kz*kz) <= kcut*kcut */
    int32_t symm;        /* 1: S of Eq. (S) (neutral electrodes); 0: S = A^-1 */
    int32_t s_prec;      /* cpm_precision of the S (v - b) product */
    int32_t k_prec;      /* cpm_precision of the b-vector sums (real and reciprocal space) */
    size_t hbm_budget;   /* bytes of device memory this context may allocate; 0 = no limit */
    int32_t chol;        /* cpm_chol of cpm_invert */
    int32_t kspace;      /* cpm_kspace of the reciprocal part of b (0: Ewald) */
    int32_t p3m_order;   /* P3M assignment order p, 2..7 (kspace = CPM_KSPACE_P3M) */
    int32_t p3m_mesh[3]; /* P3M mesh points per axis: powers of two in [8, 512]; one complex xy plane
                            (Kx Ky x 8 bytes, x 16 with k_prec = CPM_PREC_FP64) at most 128 KiB.
                            The charge assignment sums exact fixed-point integers: every charge
                            and the charge of every mesh point must stay below 2,048 e */
    int32_t p3m_matrix;  /* 1 (with kspace = CPM_KSPACE_P3M): the reciprocal part of A by the same
                            mesh operator as b, in FP64 (row i is the interpolated mesh potential of a
                            unit charge at site i; the package's pppm/electrode matrix); the xy plane
                            limit above then applies with 16 bytes per point.  0: A by the Ewald sum */
} cpm_params;

typedef struct cpm_ctx cpm_ctx;

/*
 * Create a context bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The context owns all
 * device state it allocates and frees it in cpm_destroy.
 * Errors: CPM_E_ARG for a null `p`/`out` or non-positive box, alpha, rcut or
 * kcut, or a P3M order or mesh outside the limits above; CPM_E_CUDA when no CUDA device is usable
 * (there is no CPU fallback).
 */
cpm_status cpm_create(const cpm_params* p, void* cuda_stream, cpm_ctx** out);

/* Free every device buffer of the context and the context itself.  NULL is a no-op. */
void cpm_destroy(cpm_ctx* ctx);

/*
 * Assemble the elastance matrix A (n x n, V/e) of the electrode sites
 * (Eq. coulomb, Sec. II.A; Gaussian charges of Sec. III.B):
 *   A_ij = K_E [ sum'_images (erfc(alpha r) - erfc(eta_ij r)) / r
 *               + sum_{0<|k|<=kcut} (4 pi / V) exp(-k^2/4alpha^2) / k^2 cos(k.(R_i - R_j))
 *               + delta_ij (sqrt(2) eta_i - 2 alpha) / sqrt(pi) - pi / (V alpha^2) + B_ij ],
 *   eta_ij = eta_i eta_j / sqrt(eta_i^2 + eta_j^2),
 *   B_ij = (4 pi / V) z_i z_j (slab), (2 pi / V)(x_i x_j + y_i y_j) (wire), 0 (3D).
 * xyz: device, n x 3 doubles; eta: device, n doubles (1/Angstrom, > 0);
 * group: device, n int32 in [0, n_groups) - the electrode of each site
 * (indicator matrix G of Sec. II.B).  Inputs are copied; the caller may free
 * them once the stream has passed this call.  Replaces any previous geometry.
 * Errors: CPM_E_ARG (n < 1, n_groups < 1, null pointers), CPM_E_BUDGET, CPM_E_OOM.
 */
cpm_status cpm_assemble(cpm_ctx* ctx, int64_t n, const double* xyz, const double* eta,
                        const int32_t* group, int32_t n_groups);

/*
 * Everything cpm_assemble does except the elastance matrix itself: the sites, the reciprocal
 * set, the phase tables and the real-space site chunks, and room for S.  For a context that
 * receives S from a checkpoint (cpm_import, cpm_load) instead of cpm_invert, e.g. a geometry that
 * a server evicted and admits again.  Arguments and errors as cpm_assemble; afterwards
 * cpm_invert, cpm_capacitance_ir and cpm_get_matrix(A) return CPM_E_STATE.
 */
cpm_status cpm_prepare(cpm_ctx* ctx, int64_t n, const double* xyz, const double* eta,
                       const int32_t* group, int32_t n_groups);

/*
 * Free A and the factor workspace (2 n^2 doubles) of an inverted context: only S, SG and u are
 * needed for cpm_bvec / cpm_update.  cpm_invert, cpm_capacitance_ir and cpm_get_matrix(A)
 * return CPM_E_STATE afterwards.  Synchronises the stream.  Errors: CPM_E_STATE (not inverted).
 */
cpm_status cpm_release_assembly(cpm_ctx* ctx);

/*
 * Refinement sweeps and final max-norm residual of A X = I of the last cpm_invert with
 * chol = CPM_CHOL_FP32_IR (0 and 0.0 for CPM_CHOL_FP64).  Errors: CPM_E_STATE (not inverted).
 */
cpm_status cpm_inversion_info(cpm_ctx* ctx, int32_t* sweeps, double* resid);

/*
 * Factor A = L L^T (FP64 blocked Cholesky, or FP32 with FP64 refinement: cpm_params.chol), form A^-1 and, with symm = 1, the
 * neutral capacitance matrix S = A^-1 - A^-1 e e^T A^-1 / (e^T A^-1 e)
 * (Eq. S, Sec. II.A), the electrode response SG = S G (n x N_g) and the
 * neutraliser u = A^-1 e / (e^T A^-1 e).  Synchronises the stream.
 * Errors: CPM_E_STATE (no geometry), CPM_E_NOT_SPD, CPM_E_OOM, CPM_E_CUDA.
 */
cpm_status cpm_invert(cpm_ctx* ctx);

/*
 * Electrolyte potential at every electrode site for m electrolyte
 * configurations of n_e point charges each (pad with Q = 0 charges for
 * replicas with fewer):
 *   b_i = K_E [ sum_j Q_j sum'_images (erfc(alpha r) - erfc(eta_i r)) / r
 *               + sum_k w_k Re(exp(-i k.R_i) rho(k)) - pi Q_tot / (V alpha^2) + B_i ],
 *   rho(k) = sum_j Q_j exp(i k.r_j),  w_k = (8 pi / V) exp(-k^2/4alpha^2)/k^2 (half space),
 *   B_i = (4 pi / V) z_i M_z (slab), (2 pi / V)(x_i M_x + y_i M_y) (wire), M = sum_j Q_j r_j.
 * xyz: device, (m * n_e) x 3 doubles; Q: device, m * n_e doubles;
 * b_out: device, m x n doubles.  Charges with Q == 0 are skipped.
 * Errors: CPM_E_STATE (no geometry), CPM_E_ARG, CPM_E_OOM, CPM_E_BUDGET.
 */
cpm_status cpm_bvec(cpm_ctx* ctx, int32_t m, int64_t n_e, const double* xyz, const double* Q,
                    double* b_out);

/*
 * Electrode charges q = S (G psi - b) for m electrolyte vectors, then (symm = 1)
 * the neutrality fix q <- q - u (e^T q) in FP64 and qtot = e^T q.
 * psi: device, m x n_groups doubles (electrode potentials, V); b: device, m x n
 * (the output of cpm_bvec); q_out: device, m x n; qtot_out: device, m doubles
 * (may be NULL).
 * Errors: CPM_E_STATE (not inverted), CPM_E_ARG.
 */
cpm_status cpm_update(cpm_ctx* ctx, int32_t m, const double* psi, const double* b, double* q_out,
                      double* qtot_out);

/*
 * Electrodes at prescribed total charge (constant charge method, Sec. II.C, Eq. ewise-conq).
 * qtilde: device, m x n_groups - the total charge of every electrode per replica (any values;
 * their sum is the total electrode charge).  With the capacitance matrix A^-1 the totals are
 * q~ = G^T A^-1 (G v~ - b); the call solves this for the electrode potentials v~ of each replica
 * (vtilde_out: device, m x n_groups, may be NULL) and applies them: q = A^-1 (G v~ - b), written
 * to q_out (device, m x n) with qtot_out (device, m, may be NULL) = e^T q.  The S product runs in
 * the context's s_prec; b as for cpm_update.  Asynchronous on the context stream.
 * Errors: CPM_E_STATE (not inverted), CPM_E_ARG, CPM_E_NOT_SPD (G^T A^-1 G singular).
 */
cpm_status cpm_update_ccm(cpm_ctx* ctx, int32_t m, const double* qtilde, const double* b, double* q_out,
                          double* qtot_out, double* vtilde_out);

/* Thermo-potentiostat parameters (Sec. II.D): time step dt and relaxation time tau (any one unit),
 * temperature T (K) and the target potential difference dv0 = v_1 - v_0 (V). */
typedef struct {
    double dt, tau, T, dv0;
} cpm_tp_params;

/*
 * One thermo-potentiostat step (Sec. II.D, Eq. deissenbeck) for a two-electrode context: with the
 * capacitor charge q = qcap[r] on electrode 1 (and -q on electrode 0), the effective potential
 * difference Delta v = v~_1 - v~_0 follows from the constant-charge relation of cpm_update_ccm for
 * this b; the new charge
 *   q' = q - C0 (Delta v - dv0)(1 - exp(-dt/tau)) + X_r sqrt(k_B T C0 (1 - exp(-2 dt/tau))),
 * C0 = g_1^T S g_1 (the vacuum capacitance, Sec. III.B), X: device, m standard normal numbers the
 * caller draws, is applied with the constant charge method.  qcap, X: device, m; q_out: device,
 * m x n; qcap_out: device, m (may alias qcap); dv_out: device, m (Delta v before the step, may be NULL).
 * Errors: CPM_E_STATE, CPM_E_ARG (not two electrodes, dt or tau <= 0, T < 0).
 */
cpm_status cpm_update_tp(cpm_ctx* ctx, int32_t m, const cpm_tp_params* tp, const double* qcap, const double* X,
                         const double* b, double* q_out, double* qcap_out, double* dv_out);

/*
 * Finite-field charges (Sec. II.F, Eq. cpm-ffield): q = S (v - b) with the site potentials
 * v = -dv0 zeta, zeta_i = z_i / L_z plus one for the sites of the bottom electrode (the electrode
 * of lower mean z), so that the potential difference dv0 acts across the electrolyte of a fully
 * periodic cell.  Needs CPM_BC_3D and two electrodes.  dv0: device, m; b, q_out, qtot_out as for
 * cpm_update.  The first call forms S zeta (FP64) and keeps it with S.
 * Errors: CPM_E_STATE, CPM_E_ARG (boundary, electrode count).
 */
cpm_status cpm_update_ffield(cpm_ctx* ctx, int32_t m, const double* dv0, const double* b, double* q_out,
                             double* qtot_out);

/*
 * One complete charge update from HOST buffers: copy the m * n_e charges and the
 * potentials to the device, run cpm_bvec and cpm_update, copy q and qtot back
 * and synchronise.  xyz: host, (m * n_e) x 3; Q: host, m * n_e; psi: host,
 * m x n_groups; q_out: host, m x n; qtot_out: host, m (may be NULL).
 * Host buffers may be pageable; page-locked memory gives faster copies.
 * On a context created with its own (non-default) stream the device part runs as
 * the CUDA graph of cpm_step_graph, captured once on the context's staging buffers
 * for each (m, n_e) and replayed (the graphs are kept as for cpm_step_graph).  When all
 * five host buffers are page-locked (cudaHostAlloc, cudaHostRegister, pinned torch
 * tensors) the copies are nodes of that graph as well, captured for those buffer
 * addresses: one graph launch and one synchronisation per call, and the buffers must stay
 * allocated while the context may replay the graph.  On the default stream, or while
 * cpm_profile is on, the kernels launch one by one.
 */
cpm_status cpm_step_host(cpm_ctx* ctx, int32_t m, int64_t n_e, const double* xyz, const double* Q,
                         const double* psi, double* q_out, double* qtot_out);

/*
 * cpm_bvec followed by cpm_update as one CUDA graph (device buffers as in those calls;
 * b_out receives b).  The first call for given (m, n_e, buffer addresses) reserves the
 * scratch, captures the launches on the context stream and instantiates the graph; later
 * calls with the same arguments replay it with one launch.  The context keeps up to 24
 * such graphs (least recently used replaced first); a call that has to grow the scratch drops
 * them all.  Needs a context created on a non-default stream.
 * Errors: as cpm_bvec / cpm_update; CPM_E_ARG for the default stream.
 */
cpm_status cpm_step_graph(cpm_ctx* ctx, int32_t m, int64_t n_e, const double* xyz, const double* Q,
                          const double* psi, double* b_out, double* q_out, double* qtot_out);

/*
 * Failure-detection self test (no paper counterpart): launches the tensor-core kernel once with
 * its copies switched off, so its first mbarrier wait can never complete and runs out after
 * wait_ms milliseconds (0 < wait_ms <= 10000).  Returns CPM_E_TIMEOUT when the bounded wait,
 * the device status word and the host report work; the context stays usable afterwards (its
 * status word is cleared).  Needs cpm_invert.
 */
cpm_status cpm_selftest_timeout(cpm_ctx* ctx, double wait_ms);

/*
 * Change the arithmetic of the S product (cpm_params.s_prec: CPM_PREC_FP64, CPM_PREC_FP32 or
 * CPM_PREC_BF16X3) of an inverted context without assembling again: S is kept in FP64 and in
 * FP32 after cpm_invert, and the three bf16 planes of the tensor-core product are made from the
 * FP64 S on their first use.  Drops the captured step graph.  Synchronises the stream.
 * Errors: CPM_E_ARG (not an S precision), CPM_E_STATE (not inverted).
 */
cpm_status cpm_set_s_prec(cpm_ctx* ctx, int32_t s_prec);

/*
 * Tile plan of the tensor-core S product (s_prec = CPM_PREC_BF16X3; the batched product
 * S [b_1 .. b_m] of Eq. electrode-wise, Sec. II.B, over m replicas sharing one geometry).  The
 * product runs as a persistent kernel over work items (128 sites x BN replicas x one K split);
 * the first time m replicas are used on a device with a geometry of n sites (outside stream
 * capture) every candidate plan - BN in {32, 64, 128}, two or three ring stages, split counts that
 * give 1 to 8 waves of items - is timed on the context stream and the fastest is kept for the
 * process per (device, n, m); inside a capture without a tuned plan an untimed default is used.
 * This call runs that choice when needed and reports it.  plan_out: host, 5 int32 (BN, stages,
 * K splits, CTAs, candidates timed); ms_out (may be NULL): the plan's time per product in ms
 * (negative when it was not timed).  Synchronises the stream.
 * Errors: CPM_E_STATE (not inverted, or the stream is capturing), CPM_E_ARG (other s_prec, m < 1).
 */
cpm_status cpm_gemm_plan(cpm_ctx* ctx, int32_t m, int32_t* plan_out, double* ms_out);

/*
 * Replace the kept tile plan for (this device, n, m) with plan[0..3] = (BN, stages, K splits,
 * CTAs); the built (BN, stages) pairs are (32, 2), (32, 3), (64, 2), (64, 3), (128, 2).  The
 * split count is rounded to whole 64-wide K steps per split and capped at 256 MiB of FP32
 * partial sums.  For tests and for callers that tune offline.  Synchronises the stream.
 * Errors: CPM_E_ARG (a pair that is not built, splits or CTAs < 1, too many splits), CPM_E_STATE.
 */
cpm_status cpm_gemm_set_plan(cpm_ctx* ctx, int32_t m, const int32_t* plan);

/* Wait for all work of the context and report any deferred kernel error. */
cpm_status cpm_sync(cpm_ctx* ctx);

/* Text of the last error of this context (empty when none).  Valid until the next call. */
const char* cpm_last_error(const cpm_ctx* ctx);

/* Matrices for cpm_get_matrix. */
typedef enum { CPM_MAT_A = 0, CPM_MAT_S = 1, CPM_MAT_SG = 2, CPM_MAT_U = 3 } cpm_matrix;

/*
 * Copy a context matrix into `out` (device): A (n x n, after cpm_assemble),
 * S (n x n), SG (n x n_groups, row-major) or u (n) after cpm_invert.
 * Synchronises the stream.
 */
cpm_status cpm_get_matrix(cpm_ctx* ctx, int32_t which, double* out);

/* Electrode-wise capacitance C~ = G^T S G (Sec. II.C, III.B); host out, n_groups x n_groups. */
cpm_status cpm_capacitance(cpm_ctx* ctx, double* C_out);

/*
 * The same C~ without the inverse (after cpm_assemble only): solves A X = [e, g_1 .. g_Ng] with
 * an FP32 Cholesky factor of A and FP64 iterative refinement (residuals against the FP64 A),
 * then C~_gh = g_g^T A^-1 g_h - (g_g^T A^-1 e)(g_h^T A^-1 e) / (e^T A^-1 e) (symm = 1; the
 * second term is dropped for symm = 0), as in Eq. (S) and Sec. II.C.  C_out: host,
 * n_groups x n_groups; iters_out, resid_out (may be NULL): refinement sweeps and the final
 * max-norm residual.  Allocates and frees its own work space (about 4 n^2 + 40 n (1 + N_g) bytes).
 * Errors: CPM_E_STATE, CPM_E_NOT_SPD (FP32 factor failed), CPM_E_OOM, CPM_E_BUDGET.
 */
cpm_status cpm_capacitance_ir(cpm_ctx* ctx, double* C_out, int32_t* iters_out, double* resid_out);

/*
 * Reciprocal vectors in use: writes at most `cap` integer triples (nx, ny, nz) of
 * the half-space set 0 < |k| <= kcut to host `nidx_out` and their count to
 * *nk (the full count even when it exceeds cap).  Valid after cpm_assemble.
 */
cpm_status cpm_kvectors(cpm_ctx* ctx, int32_t* nidx_out, int64_t cap, int64_t* nk);

/* Save / load S, SG and u with a header that records n, the parameters and a
 * hash of the geometry (the write_inv / read_inv files of SI Sec. 1.A).
 * Load requires cpm_assemble or cpm_prepare of the same geometry first. */
cpm_status cpm_save(cpm_ctx* ctx, const char* path);
cpm_status cpm_load(cpm_ctx* ctx, const char* path);

/*
 * The same checkpoint in caller-owned host memory (page-locked memory copies fastest).
 * cpm_export writes header + S (n x n) + SG (n x N_g) + u (n) doubles into buf (cap bytes) and
 * the size into *bytes; buf = NULL only reports the size.  cpm_import reads it back into a
 * context of the same geometry and parameters (after cpm_assemble or cpm_prepare) and marks it
 * inverted.  Both synchronise the stream.
 * Errors: CPM_E_STATE (export before cpm_invert, import before assembly), CPM_E_ARG (buffer too
 * small, or a checkpoint of another geometry or other parameters).
 */
cpm_status cpm_export(cpm_ctx* ctx, void* buf, size_t cap, size_t* bytes);
cpm_status cpm_import(cpm_ctx* ctx, const void* buf, size_t bytes);

/* Bytes of device memory currently held by the context. */
size_t cpm_device_bytes(const cpm_ctx* ctx);

/* Number of kernels the per-step calls (cpm_bvec, cpm_update, cpm_step_host) have launched. */
int64_t cpm_launch_count(const cpm_ctx* ctx);

/* Kernels that cpm_profile can time (per-step path). */
typedef enum {
    CPM_K_STATS = 0,    /* per-replica total charge and dipole */
    CPM_K_CELLS = 1,    /* cell-list binning, scan and scatter */
    CPM_K_REAL = 2,     /* real-space b */
    CPM_K_PHASES = 3,   /* electrolyte phase tables */
    CPM_K_SF = 4,       /* structure factor rho(k) */
    CPM_K_SFRED = 5,    /* structure-factor split reduction and weighting */
    CPM_K_SITE = 6,     /* reciprocal-space potential at the sites */
    CPM_K_COMBINE = 7,  /* b assembly (background, boundary term) */
    CPM_K_GEMV = 8,     /* S (G psi - b) */
    CPM_K_NEUTRAL = 9,  /* neutrality fix and total charge */
    CPM_K_COL0 = 10,    /* FP64 k_perp = 0 column of the single-precision path */
    CPM_K_TCGEMM = 11,  /* the tensor-core product alone (inside CPM_K_GEMV when s_prec = BF16X3) */
    CPM_K_P3M = 12,     /* P3M reciprocal part (assignment, transforms, interpolation) */
    CPM_K_COUNT = 13
} cpm_kernel;

/*
 * Tracing: with enable = 1 every later launch of the kernels above is bracketed
 * by CUDA events on the context stream; enable = 0 stops recording.  The events
 * stay pending until cpm_profile_read, which synchronises and returns the summed
 * device time (ms) and the launch count of one kernel since the last reset
 * (reset = 1 clears all counters after reading).
 */
cpm_status cpm_profile(cpm_ctx* ctx, int32_t enable);
cpm_status cpm_profile_read(cpm_ctx* ctx, int32_t kernel, double* total_ms, int64_t* launches, int32_t reset);

/*
 * cpm_bvec_noalloc - the electrolyte potential b of cpm_bvec for ONE electrolyte
 * configuration (FP64), computed without allocating any device memory.
 *
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot call cudaMalloc: code running inside another framework's memory pool or
 * allocator hooks, a CUDA-graph node that must not allocate, or an embedding that
 * forbids allocation after start-up.  It needs no context: the caller passes the
 * parameters, the sites (site_xyz: device, n x 3; site_eta: device, n), the charges
 * (xyz: device, n_e x 3; Q: device, n_e) and the output b_out (device, n doubles),
 * and the work is issued on `cuda_stream` (a cudaStream_t, NULL = default stream).
 *
 * Scratch: a fixed device array of 262,144 complex doubles (4 MiB) built into the
 * library, which every GPU that loads the library holds until the process exits.
 * The reciprocal-space grid, (NX + 1)(2 NY + 1)(2 NZ + 1) entries with
 * N_d = floor(kcut L_d / 2 pi) + 1, must fit in it; a larger grid returns
 * CPM_E_BUDGET and launches nothing.  Every call made outside stream capture looks
 * up the array's device address (cudaGetSymbolAddress) with the current device, so a
 * device reset between calls is harmless; a call made while `cuda_stream` is being
 * captured reuses the address of the last uncaptured call on that device, so make at
 * least one call on each device before any stream capture (CPM_E_STATE otherwise).
 * All calls share the one array, so calls whose work overlaps on the GPU (other
 * streams, other threads) race and must be serialised by the caller.  The device
 * pointers cannot be checked here: site_eta and b_out must hold n doubles, site_xyz
 * n x 3, xyz n_e x 3 and Q n_e (the Python binding checks them).  Real-space pairs
 * are summed directly over all charges and images (no cell list), so the cost grows
 * as n * n_e.
 * Errors: CPM_E_ARG (bad parameters or pointers, CPM_BC_EW2D, kspace other than
 * CPM_KSPACE_EWALD), CPM_E_BUDGET (grid too large),
 * CPM_E_STATE (first call on a device inside a stream capture), CPM_E_CUDA (no device,
 * or a launch failed).
 */
cpm_status cpm_bvec_noalloc(const cpm_params* p, int64_t n, const double* site_xyz, const double* site_eta,
                            int64_t n_e, const double* xyz, const double* Q, double* b_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* CPM_H */
