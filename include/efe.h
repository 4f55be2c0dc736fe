/*
 * efe.h -- C ABI of libefe: the orthogonalized enriched finite element (EFE)
 * Kohn-Sham eigensolver path on one GPU (sm_103a).
 *
 * The operations follow "Large-scale pseudopotential density functional
 * theory calculations using orthogonalized enriched finite element basis":
 *   Sec. II.A  Eq. (KS)                 the Kohn-Sham eigenproblem
 *   Sec. II.B  Eqs. (cutoff), (N^E)     enrichment functions, orthogonalized
 *   Sec. II.B  Eqs. (Discrete_Eig_Gen_H/M)  H^E psi = eps M^E psi, M^ec = 0
 *   Sec. III.A Eq. (MEInvApprox)        (M~^E)^-1 = diag(M^cc)^-1 + atom blocks
 *   Sec. III.B Eqs. (ChebyRecur), (residual), (residualapprox), (projectedKSEig)
 *   Sec. II.A  Eqs. (rhocompute), (electronconstraint), (EellocReform), (poisson)
 *
 * Conventions shared by every call
 *   - Every function returns efe_status; nothing throws across the ABI.
 *   - Pointers documented "device" are CUDA device pointers owned by the
 *     caller; the library never frees them.  "host" pointers are ordinary
 *     memory.  All device work is issued on the stream given to efe_setup and
 *     is finished when a call that returns host values returns; calls that
 *     return nothing on the host may still be running on that stream.
 *   - Arguments are validated before any launch; on EFE_ERR_ARG nothing ran.
 *   - efe_last_error() gives a one-line description of the last failure.
 *
 * Block-vector layout ("rows")
 *   A block of N vectors is a row-major (n_rows x ld) array of doubles, ld >= N
 *   (ld = N unless stated), with
 *     rows [0, n_nodes)           FE nodes of the full (Gx x Gy x Gz) GLL grid,
 *                                 node n = (iz*Gy + iy)*Gx + ix, G* = ncell* p + 1;
 *                                 Dirichlet boundary rows are kept and held at 0
 *     rows [n_nodes, n_rows)      enrichment coefficients, 4 per atom
 *                                 (s, px, py, pz), atom-major.
 *   Fields at quadrature points are arrays of n_cells * nq^3 doubles, cell
 *   c = (cz*ny + cy)*nx + cx, point q = (qz*nq + qy)*nq + qx, Gauss-Legendre
 *   points per axis per cell.
 */
#ifndef EFE_H
#define EFE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct efe_ctx efe_ctx; /* opaque, owned by the library */

typedef enum {
    EFE_OK = 0,
    EFE_ERR_ARG = 1,         /* invalid argument; nothing was launched */
    EFE_ERR_CUDA = 2,        /* a CUDA runtime or library call failed */
    EFE_ERR_NOT_SPD = 3,     /* an overlap block is not positive definite */
    EFE_ERR_NO_CONVERGE = 4, /* iteration cap reached before the tolerance */
    EFE_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
    EFE_ERR_OOM = 6,         /* device allocation failed */
    EFE_ERR_STATE = 7        /* call order violated (e.g. no potential set) */
} efe_status;

typedef enum {
    EFE_FP64 = 0, /* every filter operation in double precision */
    EFE_FP32 = 1, /* filter cell products and recurrence in float (FP32 accumulate) */
    EFE_BF16 = 2  /* filter cell products on tcgen05 tensor cores, bf16 operands,
                     FP32 accumulate; recurrence stored in float */
} efe_precision;

/* Uniform mesh of cubic cells of side h over [0, nx h] x [0, ny h] x [0, nz h]
 * (Sec. III.A spectral elements).  degree p in [1, 8]; nquad Gauss points per
 * axis per cell for every integral except the GLL-lumped M^cc (0 -> p + 2). */
typedef struct {
    double h;
    int ncell[3];
    int degree;
    int nquad;
} efe_mesh;

/* Atoms (Sec. II.A): positions in bohr (natoms x 3, host), valence charges. */
typedef struct {
    int natoms;
    const double *xyz;
    const double *zval;
} efe_atoms;

/* Enrichment (Sec. II.B): per atom a_s = Y00 g0 h, a_pm = r Y_1m g1 h with
 * g_l(r) = r^l exp(-alpha r^2) and the smooth cutoff h(r, r0, t), r0 chosen so
 * that the support ends at r_end: r0 = r_end t / (1 + t).  enabled = 0 gives
 * the classical FE basis alone. */
typedef struct {
    int enabled;
    double alpha;
    double r_end;
    double t;
} efe_enrichment;

/* Pseudopotential: local part v_loc = -Z erf(r / rloc) / r (enters only via
 * the Gaussian smeared charge of the electrostatics) and a separable nonlocal
 * part sum_I sum_lm |beta_Ilm> h_Il <beta_Ilm| with s and p Gaussian
 * projectors exp(-r^2/(2 rc^2)) (unit norm), truncated at r_trunc.
 * h: host, natoms x 2 (h_s, h_p) in Ha.  enabled = 0 drops the nonlocal part. */
typedef struct {
    int enabled;
    double rc;
    double r_trunc;
    const double *h;
    double rloc;
} efe_psp;

typedef struct {
    long long n_nodes;   /* FE rows incl. boundary */
    long long n_fe_dof;  /* interior FE nodes (true unknowns) */
    long long n_rows;    /* n_nodes + n_enr */
    long long n_quad;    /* n_cells * nq^3 */
    int n_enr;
    int n_proj;
    int n_cells;
    int ne;              /* (p+1)^3 nodes per cell */
    int nq;              /* Gauss points per axis */
    int grid[3];         /* Gx, Gy, Gz */
    long long n_support_nodes; /* FE nodes inside the support of at least one
                                  enrichment or projector function */
} efe_dims;

/* Timings of the last efe_chfsi / efe_filter call, from CUDA events on the
 * library stream (milliseconds), and the number of kernels it launched. */
typedef struct {
    double ms_filter;
    double ms_rr;
    double ms_lanczos;
    double ms_cell;      /* the cell-product sweeps inside the last filter */
    long long launches;  /* kernels launched by the last filter */
    long long cell_launches; /* of which cell-product kernels */
    int passes;
    double ms_rec;       /* the FE-node recurrence kernels (gather of the cell
                            products, coupling, Eq. residualapprox) inside the last
                            bf16 filter */
    long long rec_launches;
} efe_stats;

/* Build the discretisation, enrichment, orthogonalization (C = B^T (M^cc)^-1,
 * M^ee = A_ee - B^T (M^cc)^-1 B, Sec. II.B), the atom blocks of M~^ee and their
 * inverses (Eq. MEInvApprox), and the projector tables.  stream: a
 * cudaStream_t (NULL = legacy default).  Fails with EFE_ERR_NOT_SPD if an atom
 * block of M^ee is not positive definite, EFE_ERR_ARG if an enrichment or
 * projector support leaves the box.  *out receives a new context. */
efe_status efe_setup(const efe_mesh *mesh, const efe_atoms *atoms,
                     const efe_enrichment *enrich, const efe_psp *psp,
                     void *stream, efe_ctx **out);

void efe_destroy(efe_ctx *ctx);
const char *efe_last_error(const efe_ctx *ctx);
efe_status efe_get_dims(const efe_ctx *ctx, efe_dims *dims);
efe_status efe_get_stats(const efe_ctx *ctx, efe_stats *stats);

/* Assemble the potential-dependent operator (Eq. KS with v_KS = veff):
 * cell matrices H_e = 1/2 K_e + int veff N_i N_j, the raw coupling blocks
 * H^ac, H^aa and, with enrichment, the blocks of H^E the mixed filter uses
 * (E = H^ac - C H^cc, H^E_ee = H^aa - C H^ca - E C^T, FP64).  veff_q: device,
 * n_quad doubles at the Gauss points.  Must be called before any H product. */
efe_status efe_set_potential(efe_ctx *ctx, const double *veff_q);

/* Y = H^E X = T^T H_raw T X (Eq. Discrete_Eig_Gen_H).  X, Y: device, rows x N,
 * not aliased.  prec selects the arithmetic of the cell products (EFE_FP64:
 * double; EFE_FP32 / EFE_BF16: inputs rounded, FP32 accumulate), used by the
 * parity tests of the tensor-core cell products.  The bf16 product keeps the
 * transform form: for vectors with large orthogonalized coordinates (such as
 * M~^-1 Z when the enrichment is nearly in the FE space) its relative error
 * grows with the cancellation; efe_filter applies the block form instead. */
efe_status efe_apply_h(efe_ctx *ctx, const double *X, double *Y, int N, efe_precision prec);

/* Y = M^E X with the exact M^E (diagonal M^cc, full M^ee). device, rows x N. */
efe_status efe_apply_m(efe_ctx *ctx, const double *X, double *Y, int N);

/* Y = (M~^E)^-1 X (Eq. MEInvApprox).  device, rows x N. */
efe_status efe_apply_minv(efe_ctx *ctx, const double *X, double *Y, int N);

/* k-step Lanczos for M~^-1 H^E in the M~ inner product from the device vector
 * u0 (rows doubles).  out (host): theta_min, theta_max, theta_max + |beta_k s_k|. */
efe_status efe_lanczos(efe_ctx *ctx, const double *u0, int k, double out[3]);

/* One residual Chebyshev filter of degree m (Eqs. residual, residualapprox
 * with the recurrence re-derived from Eq. ChebyRecur):
 *   G = HV - M^E V diag(lam);  Z_1 = (s1/e) G;
 *   Z_k = (2 s_k/e)(H M~^-1 Z_{k-1} - c Z_{k-1}) - s_{k-1} s_k Z_{k-2}
 *         + (2 s_k/e) G diag(C_{k-1}(lam));
 *   Vout = M~^-1 Z_m + V diag(C_m(lam)).
 * V, HV, Vout: device rows x N (HV = H^E V in double); lam: device N doubles;
 * bounds (host): a0 <= lowest wanted, [a, b] the damped interval.  With
 * prec = EFE_BF16 the products inside the recurrence apply H^E through its
 * blocks (E = H^ac - C H^cc, H^E_ee = H^aa - C H^ca - E C^T and the projector
 * overlaps P^E = P_a - P_c C^T, assembled in FP64 by efe_set_potential and
 * setup) rather than as T^T H_raw T, whose two terms cancel when the
 * enrichment is nearly representable by the FE space.  In bf16 the FE rows of
 * the recurrence are carried as Y_k = M~^-1 Z_k (and G as M~^-1 G) in bf16
 * storage -- Y_k is the operand of the next cell products -- with FP32
 * arithmetic; the storage rounding scales with the residual like that of the
 * operands.  The enriched rows keep Z_k in FP32.  EFE_BF16 takes up to 256
 * columns per pass; wider blocks are filtered in balanced column blocks
 * (gathered, filtered, scattered back; the filter of each column is
 * independent of the others). */
efe_status efe_filter(efe_ctx *ctx, const double *V, const double *HV, const double *lam,
                      int N, int m, const double bounds[3], efe_precision prec, double *Vout);

/* Storage of the per-cell products H_e Y_e inside the bf16 filter before the
 * per-node sums: EFE_BF16 (the default; half the memory traffic of that
 * round trip) or EFE_FP32.  Both accumulate in FP32 on the tensor cores and
 * sum in FP32.  Not a part of the paper's method: a precision knob of this
 * implementation.  EFE_ERR_ARG for other values. */
efe_status efe_set_cell_storage(efe_ctx *ctx, efe_precision prec);

/* How the Poisson solves (efe_poisson and those inside efe_scf) iterate:
 * EFE_FP64 -- conjugate gradients in FP64; EFE_FP32 -- iterative refinement:
 * the residual and the solution in FP64, the correction equations by FP32
 * conjugate gradients (each to 1e-4 of its right-hand side), then an FP64
 * check; the stopping test is the FP64 residual either way, so both meet the
 * same tolerance.  Default (until this is called): EFE_FP32 on meshes of
 * 2^20 nodes or more (where the FP64 operator dominates), else EFE_FP64.  Not
 * a part of the paper's method.  EFE_ERR_ARG for other values. */
efe_status efe_set_poisson_precision(efe_ctx *ctx, efe_precision prec);

/* Rayleigh-Ritz with the exact M^E (Eq. projectedKSEig), in place:
 * X <- X D, HX <- H^E X D with D^T (X^T M X) D = I, ascending eigenvalues.
 * X, HX: device rows x N (HX is computed here); eig, resid: host N doubles
 * (resid_i = ||H psi_i - eps_i M psi_i||_2).  EFE_ERR_NOT_SPD if X^T M X is
 * not positive definite (dependent columns) or the generalized eigensolve
 * fails. */
efe_status efe_rayleigh_ritz(efe_ctx *ctx, double *X, double *HX, int N,
                             double *eig, double *resid);

/* Multipass residual ChFSI (Sec. III.B): Rayleigh-Ritz on X, then passes of
 * efe_filter + Rayleigh-Ritz until max(resid[0:nconv]) < tol or max_pass.
 * bounds (host, a0, a, b) or NULL for a 10-step Lanczos from u0 (device)
 * with a0 = theta_min, a = a0 + 0.3 (b - a0); later passes a = max Ritz value,
 * a0 = min Ritz value.  X, HX: device rows x N, in/out (HX may be NULL).
 * eig, resid: host N.  passes: host, may be NULL.  EFE_ERR_NO_CONVERGE when
 * max_pass is reached (results are still written).  With prec = EFE_BF16 the
 * passes run in bf16 while each reduces max(resid[0:nconv]); after one that
 * does not, the remaining passes run in FP32. */
efe_status efe_chfsi(efe_ctx *ctx, double *X, double *HX, int N, int m, const double *bounds,
                     const double *u0, int max_pass, double tol, int nconv,
                     efe_precision prec, double *eig, double *resid, int *passes);

/* The standard Chebyshev filter with the approximate inverse (Eq. ChebyRecur
 * applied to A = M~^-1 H^E, the method the residual filter replaces; Sec. III.B,
 * Fig. 1): Vout = C_m(M~^-1 H^E) V by
 *   Y_0 = V;  Y_1 = (s1/e)(M~^-1 H V - c V);
 *   Y_k = (2 s_k/e)(M~^-1 H Y_{k-1} - c Y_{k-1}) - s_{k-1} s_k Y_{k-2},
 * run in the variables Z_k = M~ Y_k so that it shares every kernel of the
 * residual filter (no forcing term, Z_0 = M~ V, Vout = M~^-1 Z_m).  Its fixed
 * points are eigenvectors of M~^-1 H^E, not of (H^E, M^E), and its rounding
 * error scales with V rather than with the residual.  Arguments as for
 * efe_filter (no Ritz values). */
efe_status efe_filter_standard(efe_ctx *ctx, const double *V, const double *HV, int N, int m,
                               const double bounds[3], efe_precision prec, double *Vout);

/* efe_chfsi with a choice of filter and a per-pass record:
 * kind = EFE_FILTER_RESIDUAL or EFE_FILTER_STANDARD, optionally or-ed with
 * EFE_FILTER_KEEP_PRECISION (bf16 passes stay bf16: no switch to FP32 after
 * a pass that does not reduce the residual).  history: host max_pass doubles
 * or NULL; entry j is max(resid[0:nconv]) after pass j + 1.  Other arguments
 * and errors as for efe_chfsi (EFE_ERR_ARG for unknown kind bits). */
enum { EFE_FILTER_RESIDUAL = 0, EFE_FILTER_STANDARD = 1, EFE_FILTER_KEEP_PRECISION = 2 };
efe_status efe_chfsi_kind(efe_ctx *ctx, double *X, double *HX, int N, int m, const double *bounds,
                          const double *u0, int max_pass, double tol, int nconv, efe_precision prec,
                          int kind, double *eig, double *resid, int *passes, double *history);

/* Same filter with host buffers (V, HV, Vout: host rows x N; lam: host N):
 * copies in, filters, copies out on the library stream, returns when done.
 * The device copies (3 rows x N + N doubles) stay allocated in the context
 * for later calls; page-locked host buffers give the full copy bandwidth. */
efe_status efe_filter_host(efe_ctx *ctx, const double *V, const double *HV, const double *lam,
                           int N, int m, const double bounds[3], efe_precision prec,
                           double *Vout);

/* ------------------------------------------------------------------------
 * Self-consistent field (Sec. II.A; Sec. IV: 500 K smearing, Anderson mixing)
 * ------------------------------------------------------------------------ */

/* b_sm at the quadrature points: sum_I -Z_I g_rloc(x - R_I), the Gaussian
 * charge whose potential is the local part -Z erf(r/rloc)/r (Eq. EZZbmsear).
 * b_q: device, n_quad. */
efe_status efe_smeared_charge(efe_ctx *ctx, double *b_q);

/* Superposition of atomic Gaussians Z_I (kappa/pi)^3/2 exp(-kappa r^2) at the
 * quadrature points, scaled so that its integral is N_e.  rho_q: device. */
efe_status efe_atomic_density(efe_ctx *ctx, double kappa, double *rho_q);

/* rho(x_q) = 2 sum_i occ_i psi_i(x_q)^2 (Eq. rhocompute) with psi the EFE
 * expansion of column i of X (device rows x N); occ: host N; rho_q: device. */
efe_status efe_density(efe_ctx *ctx, const double *X, int N, const double *occ, double *rho_q);

/* LDA exchange-correlation (Slater + Perdew-Wang 1992, spin-unpolarised) at
 * every quadrature point; densities below 1e-14 give 0.  Either output may be
 * NULL.  All device, n_quad. */
efe_status efe_xc(efe_ctx *ctx, const double *rho_q, double *vxc_q, double *exc_q);

/* FE solution of -1/(4 pi) Lap phi = f with phi = 0 on the box (Eq. poisson),
 * Jacobi-preconditioned conjugate gradients to ||r|| < tol ||F|| (the FP64
 * residual; see efe_set_poisson_precision for how the iterations run).
 * f_q: device n_quad; phi_nodes: device n_nodes (out); phi_q: device n_quad
 * (out, may be NULL); iters, rel_res: host (may be NULL). */
efe_status efe_poisson(efe_ctx *ctx, const double *f_q, double *phi_nodes, double *phi_q,
                       double tol, int max_it, int *iters, double *rel_res);

/* Fermi level mu with 2 sum_i f(eig_i, mu) = n_elec (Eq. electronconstraint),
 * f = 1/(1 + exp((eig - mu)/kT)), by bisection on the GPU.  eig, occ: host N. */
efe_status efe_fermi(efe_ctx *ctx, const double *eig, int N, double n_elec, double kT,
                     double *mu, double *occ);

/* *out = int a b (quadrature), b may be NULL (int a).  a_q, b_q: device. */
efe_status efe_integrate(efe_ctx *ctx, const double *a_q, const double *b_q, double *out);

/* *out = int a b, like efe_integrate, without allocating any device memory:
 * for callers that cannot call cudaMalloc while they run (code whose device
 * memory belongs to another allocator, or a host that must not grow device
 * memory after start-up).  The paper has no counterpart; this is a library
 * service.  The per-cell partial sums go to a fixed array in the library's
 * device memory, sized for at most 65,536 cells (512 KB, held by every GPU
 * that loads the library until the process exits); larger meshes get
 * EFE_ERR_ARG.  The call runs on the device the context was made on (made
 * current for the call, the caller's device restored after).  The first call
 * on a device looks the array's address up with that device current and
 * caches it for the life of the process (the lookup is thread-safe), so make
 * that first call before any stream capture.  Every call shares the array:
 * calls that overlap on the GPU (several streams, several contexts on one
 * device) race; serialise them.  Nothing in the array needs to start at
 * zero: each call overwrites what it reads.  a_q, b_q: device n_quad (b_q may
 * be NULL); out: host. */
efe_status efe_integrate_noalloc(efe_ctx *ctx, const double *a_q, const double *b_q, double *out);

typedef void (*efe_scf_log_fn)(void *user, int iter, double E, double F, double mu,
                               double drho, double dE, double resid0);

typedef struct {
    int cheb_degree;      /* filter degree m */
    double temperature;   /* smearing temperature, K */
    double mix_beta;      /* Anderson mixing parameter */
    int mix_history;      /* Anderson history length, 0..8 */
    double tol_rho;       /* ||rho_out - rho_in||_L2 / N_e */
    double tol_e;         /* |E_k - E_{k-1}| per atom, Ha */
    int max_iter;
    double first_tol;     /* first iteration: passes until the max residual of the
                             occupied states is below this */
    int first_max_pass;
    int renormalize;      /* scale rho_out to integrate to N_e */
    double kappa;         /* exponent of the atomic Gaussians of the start density */
    double poisson_tol;
    int precision;        /* efe_precision of the filter passes */
    efe_scf_log_fn log;   /* optional per-iteration callback */
    void *log_user;
    double bf16_resid;    /* with precision EFE_BF16: the passes of the first iteration
                             run in bf16; a later pass runs in bf16 while the largest
                             residual of the occupied states after the last
                             Rayleigh-Ritz exceeds this, in FP32 below it (0: every
                             pass in bf16, the binding's default) */
    int profile;          /* nonzero: synchronise at phase ends and report the
                             phase times in efe_scf_result.ms_phase */
    int passes;           /* filter passes (each followed by Rayleigh-Ritz) per
                             iteration after the first; values below 1 mean 1 */
    double precond_k2;    /* > 0: Kerker preconditioning of the Anderson step (not in
                             the paper, whose mixing is plain Anderson): the mixed
                             residual Rbar enters as Rbar - k2 (-Lap + k2)^-1 Rbar,
                             the inverse by CG on the FE mesh (lumped mass, phi = 0
                             on the box); bohr^-2.  0: plain Anderson. */
} efe_scf_opts;

typedef struct {
    double E;             /* total energy (Ha) */
    double F;             /* free energy E - TS */
    double mu;            /* Fermi level */
    double drho, dE;      /* last convergence measures */
    int iters, converged;
    long long poisson_iters;
    double *eig;          /* host N (optional, caller-owned) */
    double *rho_q;        /* device n_quad (optional, caller-owned): final rho_out */
    double ms_phase[5];   /* with opts.profile: wall time of the potential (Poisson, XC,
                             operator assembly), the eigensolver (Lanczos, filter,
                             Rayleigh-Ritz), the density (Fermi level, rho_out), the
                             energy (Poisson of rho_out, integrals) and the mixing */
} efe_scf_result;

/* The SCF loop: v_eff = v_xc[rho_in] + phi[rho_in + b_sm]; operator assembly;
 * eigenpairs by residual ChFSI (first iteration: Lanczos bounds and passes
 * until first_tol; later: opts.passes filter passes, each with Rayleigh-Ritz);
 * Fermi level;
 * rho_out; E = 2 sum f eps - int rho_out v_eff + E_xc[rho_out]
 * + 1/2 int (rho_out + b) phi[rho_out] - E_self + dE_ZZ; Anderson mixing.
 * X: device rows x N, start vectors in, eigenvectors out; u0: device rows
 * (Lanczos start); rho0_q: device n_quad or NULL (atomic superposition).
 * EFE_ERR_NO_CONVERGE after max_iter (results still written). */
efe_status efe_scf(efe_ctx *ctx, const efe_scf_opts *opts, double *X, int N, const double *u0,
                   const double *rho0_q, efe_scf_result *res);


/* ------------------------------------------------------------------------
 * Learned density warm start.  The paper starts the SCF from a superposition
 * of atomic densities (Sec. II.A, Sec. IV); the learned correction on top of
 * it is an addition of this library, with the superposition as its fallback
 * and the converged SCF as the measure of its worth.
 *
 *   descriptors  D_Ik = sum_{J != I, r_IJ < 10} Z_J exp(-(r_IJ - mu_k)^2 / 0.32)
 *                       * (1 + cos(pi r_IJ / 10)) / 2,   mu_k = 2 + 8 k / 31,
 *                k = 0..31, lengths in bohr (computed in double, stored float)
 *   network      x = (D - x_mean) / x_std; three hidden layers of 128 SiLU units
 *                (silu(z) = z / (1 + e^-z)); linear output y (8);
 *                coefficients c = y_mean + y_std * y.  Float arithmetic.
 *   correction   drho(x) = sum_I sum_k c_Ik phi_k(|x - R_I|), zero beyond 8 bohr;
 *                phi = L^-1 g, the per-atom orthonormal combinations of the
 *                normalised Gaussians g_j(r) = (kappa_j/pi)^{3/2} exp(-kappa_j r^2),
 *                kappa_j = 0.5 * 16^{j/7} (j = 0..7), S = L L^T, S = int g g^T.
 *   warm start   rho_0 = max(rho_sup + drho, 0) scaled to N_e.
 *   training     loss = mean over samples and outputs of (y - (c* - y_mean)/y_std)^2,
 *                c* the least-squares coefficients of rho_scf - rho_sup
 *                (efe_fit_correction); full-batch Adam.
 *
 * Parameter vector theta: EFE_MLP_N_PARAMS floats, device, caller-owned:
 *   W1[128][32] b1[128] W2[128][128] b2[128] W3[128][128] b3[128] W4[8][128] b4[8]
 *   (EFE_MLP_N_TRAIN trained values, weights row-major [out][in]), then
 *   x_mean[32] x_std[32] y_mean[8] y_std[8] (set by efe_mlp_normalise).
 * Samples are rows: D is n x 32, targets T and coefficients C are n x 8 (floats).
 * ------------------------------------------------------------------------ */
#define EFE_MLP_N_DESC 32
#define EFE_MLP_N_OUT 8
#define EFE_MLP_N_TRAIN 38280
#define EFE_MLP_N_PARAMS 38360

typedef struct efe_mlp efe_mlp; /* opaque: training workspace, owned by the library */

typedef struct {
    float lr, beta1, beta2, eps;   /* Adam (Kingma & Ba 2015) step size and decay rates */
} efe_adam;

/* Workspace for training on up to max_samples samples at a time, working on
 * `stream` (a cudaStream_t; NULL = the default stream).  Training steps are
 * replayed from a CUDA graph captured on a private stream that is ordered
 * after, and before, the given stream. */
efe_status efe_mlp_create(void *stream, int max_samples, efe_mlp **out);
void efe_mlp_destroy(efe_mlp *mlp);
/* Last failure of a call on this workspace (NULL: of efe_mlp_create). */
const char *efe_mlp_last_error(const efe_mlp *mlp);

/* Descriptors of n atoms.  xyz: device n x 3 (bohr); zval: device n; D: device
 * n x 32 (out). */
efe_status efe_descriptors(efe_mlp *mlp, const double *xyz, const double *zval, int n, float *D);

/* C = network(D) in physical units.  theta: device; D: device n x 32; C: device
 * n x 8 (out).  Any n >= 0. */
efe_status efe_mlp_forward(efe_mlp *mlp, const float *theta, const float *D, int n, float *C);

/* Sets x_mean, x_std (floor 1e-2), y_mean, y_std (floor 1e-8) of theta to the
 * per-column mean and standard deviation of D and T (n samples, device). */
efe_status efe_mlp_normalise(efe_mlp *mlp, float *theta, const float *D, const float *T, int n);

/* Loss of the normalised outputs against targets T (device n x 8) and its
 * gradient (device EFE_MLP_N_TRAIN, out) by back-propagation; loss: host.
 * 1 <= n <= max_samples.  Per-CTA partial gradients are summed in a fixed
 * order, so repeated calls give identical bits. */
efe_status efe_mlp_loss_grad(efe_mlp *mlp, const float *theta, const float *D, const float *T, int n,
                             float *grad, double *loss);

/* One Adam update of the trained part of theta with gradient grad (device),
 * step number t >= 1; m, v: device EFE_MLP_N_TRAIN moments (start at zero). */
efe_status efe_mlp_adam(efe_mlp *mlp, float *theta, float *m, float *v, const float *grad, int t,
                        const efe_adam *hp);

/* `steps` full-batch Adam steps numbered t0+1 .. t0+steps on (D, T): each step
 * is the loss/gradient pass and the update, replayed from one CUDA graph.
 * loss_hist: device `steps` floats (out), the loss before each update. */
efe_status efe_mlp_train(efe_mlp *mlp, float *theta, float *m, float *v, const float *D, const float *T,
                         int n, int steps, int t0, const efe_adam *hp, float *loss_hist);

/* Parameter file: the 8-byte tag "EFEMLP01", the count EFE_MLP_N_PARAMS as a
 * little-endian int32, then the floats of theta (little-endian).  theta:
 * device.  efe_mlp_load fails with EFE_ERR_ARG (nothing written to theta) if
 * the file is missing, truncated or carries another tag or count. */
efe_status efe_mlp_save(efe_mlp *mlp, const float *theta, const char *path);
efe_status efe_mlp_load(efe_mlp *mlp, const char *path, float *theta);

/* drho at the quadrature points of ctx's mesh from coefficients c (device
 * natoms x 8, atom order of efe_setup).  drho_q: device n_quad (out). */
efe_status efe_density_correction(efe_ctx *ctx, const double *c, double *drho_q);

/* Least-squares coefficients of the density difference drho = rho_q - base_q
 * (device n_quad each; base_q may be NULL for drho = rho_q):
 * (Phi^T W Phi + ridge I) c = Phi^T W drho, W the quadrature weights, Phi the
 * phi_Ik at the quadrature points (Gram matrix by the same quadrature; FP64,
 * Cholesky).  c: device natoms x 8 (out).  EFE_ERR_NOT_SPD if the system is
 * not positive definite (ridge = 0 with dependent functions). */
efe_status efe_fit_correction(efe_ctx *ctx, const double *rho_q, const double *base_q, double ridge, double *c);

/* The superposition (as efe_atomic_density with kappa) plus the correction
 * with coefficients c (device natoms x 8), clipped at zero and scaled to N_e;
 * the superposition alone when that density is not finite or has no charge.
 * rho_q: device n_quad (out); fallback: host (may be NULL), 1 when rho_q is the
 * superposition. */
efe_status efe_corrected_density(efe_ctx *ctx, const double *c, double kappa, double *rho_q, int *fallback);

/* Start density: the superposition (as efe_atomic_density with kappa) plus the
 * network's correction, clipped at zero and scaled to N_e.  theta: device
 * parameters, or NULL for the superposition alone.  The superposition is also
 * returned when the corrected density has no positive charge or is not finite.
 * rho_q: device n_quad (out); fallback: host (may be NULL), 1 when rho_q is the
 * superposition. */
efe_status efe_warm_start(efe_ctx *ctx, efe_mlp *mlp, const float *theta, double kappa, double *rho_q,
                          int *fallback);

#ifdef __cplusplus
}
#endif
#endif /* EFE_H */
