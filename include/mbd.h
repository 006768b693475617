/*
 * mbd.h - C ABI of the GB300 SPME stochastic-Lanczos MBD library.
 *
 * Method: arXiv 2307.02278 (Poier, Lagardere, Piquemal), "Smooth Particle Mesh
 * Ewald-integrated stochastic Lanczos Many-body Dispersion algorithm".
 *
 *   E_MBD = (1/2) Tr sqrt(C) - (3/2) sum_i w_i                       (Eq. plasmonic2)
 *   C     = Omega + Diag(g) T'^pbc Diag(g),  Omega = (+)_i w_i^2 I_3,
 *           g = (+)_i w_i sqrt(alpha_i) 1_3                          (Eqs. ccd, gvec, lk3)
 *   T'^pbc d = E^dir + E^rec + E^self by Ewald summation, tin-foil boundary,
 *           with E^rec from SPME                                      (Eqs. ewalddip, fld_ewald,
 *                                                                      fld_ewald1, spme, dipolarr)
 *   Tr sqrt(C) ~ (3N/R) sum_l sum_k U_1k^2 sqrt(theta_k) over R Rademacher
 *           probes and an m-step Lanczos recurrence per probe        (Eqs. hutch, dds, recurs2,
 *                                                                      sl4; Algorithms 1 and 2)
 *
 * Units: atomic units throughout (bohr, hartree, bohr^3).
 *
 * Conventions for every entry point:
 *   - Every call returns an mbd_status; nothing aborts or throws across the ABI.
 *     Output buffers are left untouched when a call fails before its GPU work
 *     starts (argument errors); after a CUDA error their contents are undefined.
 *   - Host pointers are read during the call only; the library keeps copies.
 *     Device pointers ("_dev") are borrowed for the duration of the call only
 *     and must be device memory of the current CUDA device.
 *   - All GPU work of a system is enqueued on the stream given at creation;
 *     every call returns after that work has finished (it synchronises the
 *     stream), so host outputs are valid on return.
 *   - A system handle is not thread-safe: one handle per host thread/stream.
 *   - Probe rule (part of the ABI, so that any implementation draws the same
 *     probes): u_{l,i} = +1 when the top bit of SplitMix64(seed + (l << 32) + i)
 *     is 0, else -1; v_l = u_l / sqrt(3N) (Eq. dds).  SplitMix64(x) is the first
 *     output of Steele, Lea & Flood's SplitMix64 generator started at state x.
 *   - The library sizes its device memory itself (cudaMalloc), growing it on
 *     demand; MBD_ERR_OOM is returned when an allocation fails.
 */
#ifndef MBD_H
#define MBD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MBD_OK = 0,
    MBD_ERR_INVALID_ARG = 1,            /* a null pointer, a size or parameter out of range */
    MBD_ERR_OOM = 2,                    /* a device or pinned-host allocation failed */
    MBD_ERR_CUDA = 3,                   /* a CUDA runtime call or kernel launch failed */
    MBD_ERR_NOT_POSITIVE_DEFINITE = 4,  /* a Ritz value of C was <= 0 (polarisation catastrophe) */
    MBD_ERR_NONFINITE = 5,              /* a NaN or Inf appeared in a result */
    MBD_ERR_TIMEOUT = 6,                /* a bounded device-side wait ran out (reserved: no kernel of
                                           this build waits on another, so no call returns it) */
    MBD_ERR_UNSUPPORTED = 7,            /* valid request this build does not support */
    MBD_ERR_NO_DEVICE = 8               /* no CUDA device is visible */
} mbd_status;

/* Arithmetic of the operator C (spreading, FFT, influence function, gather,
 * real-space field).  The Lanczos vectors, dot products, the quadrature of
 * the tridiagonal and the trace sum are always FP64. */
enum { MBD_FP64 = 0, MBD_MIXED = 1 /* FP32 operator, FP64 Lanczos */ };

/* Evaluation of each probe's Gauss quadrature (Eqs. tridiag2, sl3):
 * q_l = sum_k U_1k^2 sqrt(theta_k) = e_1^T Delta^{1/2} e_1, and for the forces
 * c = U diag(theta^{-1/2}) U^T e_1 = Delta^{-1/2} e_1.
 *   MBD_QUAD_CHEBYSHEV (default, FP64): both from a Chebyshev expansion of
 *     sqrt(x) and 1/sqrt(x) on an interval that contains the spectrum of Delta
 *     (Gershgorin above, Sturm-count multisection below), applied to e_1 by the
 *     three-term recurrence.  These are the same quantities as the
 *     eigendecomposition route, to about 1e-13.  A probe whose Delta is too
 *     ill-conditioned for 256 terms is done by QL.
 *   MBD_QUAD_QL: the implicit-QL eigendecomposition of Delta (the paper's
 *     route), FP64.
 *   MBD_QUAD_QL_DF64: the same QL in double-float arithmetic (pairs of FP32
 *     numbers, 48-bit significand; about 1e-13 from FP64).
 * A Ritz value <= 0 gives MBD_ERR_NOT_POSITIVE_DEFINITE with every method. */
enum { MBD_QUAD_CHEBYSHEV = 0, MBD_QUAD_QL_DF64 = 1, MBD_QUAD_QL = 2 };

/* Field terms for mbd_field (bit mask). */
enum { MBD_TERM_REAL = 1, MBD_TERM_RECIP = 2, MBD_TERM_SELF = 4, MBD_TERM_ALL = 7 };

typedef struct mbd_system mbd_system;   /* opaque, owned by the library */
typedef struct mbd_batch mbd_batch;     /* opaque: several independent systems */

/* One periodic system (Eq. ham parameters, Ewald/SPME settings).
 * damping: T'_ij = s(R_ij) T_ij with the Fermi form
 *   s(r) = 1 / (1 + exp(-damp_d (r / (damp_beta (Rvdw_i + Rvdw_j)) - 1)))
 * (the paper defers the explicit damping to its earlier SL-MBD work).
 * Real space: the erfc-screened field is summed over image pairs with
 * |r| < r_cut and the damping correction -(1-s) T over |r| < damp_cut
 * (Eq. fld_ewald); damp_cut <= 0 means damp_cut = r_cut. */
typedef struct {
    int32_t n_atoms;          /* N >= 1 */
    double cell[9];           /* rows a1, a2, a3 (bohr), right-handed (det > 0) */
    const double *pos;        /* host [N][3] Cartesian (bohr); wrapped into the cell */
    const double *alpha;      /* host [N] static polarisability (bohr^3), > 0 */
    const double *omega;      /* host [N] characteristic frequency (Ha), > 0 */
    const double *r_vdw;      /* host [N] vdW radius (bohr), > 0 */
    double damp_beta;         /* Fermi range-separation parameter, > 0 */
    double damp_d;            /* Fermi steepness, > 0 */
    double ewald_beta;        /* Ewald splitting parameter (bohr^-1), > 0 */
    double r_cut;             /* real-space cutoff (bohr), > 0 */
    double damp_cut;          /* damping-correction cutoff (bohr); <= 0: = r_cut */
    int32_t mesh[3];          /* K_alpha: products of 2, 3, 5 only; 2p <= K_alpha <= 1000 */
    int32_t spline_order;     /* p: even, 4 <= p <= 10 */
    int32_t precision;        /* MBD_FP64 or MBD_MIXED */
    int32_t quadrature;       /* MBD_QUAD_CHEBYSHEV (default), MBD_QUAD_QL or MBD_QUAD_QL_DF64 */
} mbd_system_desc;

/* Create a system: validate, upload, build the neighbour list, spline
 * stencils, the influence function and the FFT tables (Algorithm 1, grid
 * allocation and neighbour list).  cuda_stream: a cudaStream_t or NULL for the
 * legacy default stream.  *out receives the handle on MBD_OK. */
mbd_status mbd_create_system(const mbd_system_desc *desc, void *cuda_stream, mbd_system **out);

/* Release all device and host memory of a system (NULL is ignored). */
void mbd_destroy_system(mbd_system *sys);

/* New positions (host [N][3], bohr) for the same atoms and cell; rebuilds the
 * neighbour list and spline stencils. */
mbd_status mbd_update_positions(mbd_system *sys, const double *pos);

/* y = C x for a block of vectors (Eqs. ccd, lk3): x_dev, y_dev are device
 * FP64 arrays of layout [nvec][N][3], nvec >= 1; y_dev may not alias x_dev. */
mbd_status mbd_apply_C(mbd_system *sys, int32_t nvec, const double *x_dev, double *y_dev);

/* Stochastic Lanczos MBD energy (Algorithm 1 with Algorithm 2 per step).
 * n_probes R >= 1, n_steps m in [1, 128] (m = size of the tridiagonal Delta).
 * Outputs (host; energy required, the rest may be NULL):
 *   energy    E_MBD (Ha)
 *   trace     the estimate of Tr sqrt(C)
 *   q_host    [R] per-probe quadrature v_l^T sqrt(C) v_l
 *   ab_host   [R][2][m]: Delta's diagonal a_1..a_m, then the couplings
 *             b_2..b_m followed by a 0 (b after a breakdown is 0)
 * Returns MBD_ERR_NOT_POSITIVE_DEFINITE if a Ritz value is <= 0. */
mbd_status mbd_lanczos_energy(mbd_system *sys, int32_t n_probes, int32_t n_steps, uint64_t seed,
                              double *energy, double *trace, double *q_host, double *ab_host);

/* Energy and forces F = -dE/dR (Ha/bohr).  The paper computes energies only
 * and names gradients as future work (Conclusions); the estimator used here is
 * dE/dR ~ (1/4)(3N/R) sum_l (g.w_l)^T (dT'/dR) (g.v_l) with w_l = C^{-1/2} v_l
 * from the Lanczos basis of probe l, on the same probes as the energy.
 * forces_dev: device FP64 [N][3].  Other arguments as mbd_lanczos_energy. */
mbd_status mbd_energy_forces(mbd_system *sys, int32_t n_probes, int32_t n_steps, uint64_t seed,
                             double *energy, double *forces_dev);

/* ---- self-consistent screening of the polarisabilities (front end) ----
 * The paper's review of the MBD model notes that the atomic polarisabilities
 * can be screened by a Dyson-like equation solved at a set of frequencies, and
 * keeps that step out of its scope: the SPME-Lanczos algorithm takes screened
 * and unscreened parameters alike.  This call computes the screened
 * parameters of the range-separated scheme for the system's atoms, geometry
 * and damping (beta, d, R_vdw):
 *   alpha_i(iu) = alpha_i / (1 + (u/omega_i)^2),
 *   sigma_i(u) = (sqrt(2/pi) alpha_i(iu)/3)^(1/3),
 *   T_SR_ij(u) = sum'_n (1 - s(|r+n|)) T_GG(r+n; sqrt(sigma_i^2 + sigma_j^2)) over
 *     |r+n| < damp_cut (the truncation of the damping correction), with
 *     T_GG(r; w) = grad_i grad_j erf(|r|/w)/|r| and s the Fermi damping,
 *   (A(u)^-1 + T_SR(u)) X_c = 1_c for c = x, y, z, A = diag(alpha_i(iu)),
 *   alpha_i^SCS(iu) = (1/3) sum_c X_c[i, c],
 *   C6_i = (3/pi) int_0^inf alpha_i^SCS(iu)^2 du over n_freq Gauss-Legendre
 *     nodes t mapped to u = 0.5 (1 + t)/(1 - t) Ha,
 *   omega_i^SCS = 4 C6_i / (3 alpha_i^SCS(0)^2),
 *   R_vdw,i^SCS = R_vdw,i (alpha_i^SCS(0) / alpha_i)^(1/3).
 * The solves are a conjugate-gradient iteration per (direction, frequency)
 * column with the preconditioner A(u), T_SR in the system's operator precision
 * (FP32 for MBD_MIXED, FP64 for MBD_FP64) and FP64 vectors; it stops when
 * every column's residual norm is at most tol sqrt(N) (tol relative to the
 * right-hand side) or after max_iter steps.  A system with screened
 * parameters is then made with mbd_create_system; its forces are the gradient
 * at fixed parameters (the dependence of alpha^SCS on positions is not
 * included).
 *   n_freq: 1..31 quadrature nodes; tol > 0; max_iter >= 0 (0: the unscreened
 *   starting point).
 *   alpha_out, omega_out, r_vdw_out: host [N] (required); c6_out: host [N] or
 *   NULL; alpha_iu_out: host [n_freq + 1][N] (static first, then the nodes in
 *   ascending u) or NULL; iterations, residual: host scalars or NULL
 *   (iterations taken, largest relative residual at exit).
 * Device memory for the call (MBD_MIXED: a 16-byte record per neighbour pair,
 * T_SR evaluated inside every product; MBD_FP64: the pair tensors, nnz x 32 x 6
 * values; and a few N x 288 FP64 vectors) is allocated and released inside it.  Errors:
 * MBD_ERR_INVALID_ARG (arguments), MBD_ERR_NOT_POSITIVE_DEFINITE (a column with
 * p.(A^-1 + T_SR)p <= 0: the polarisation catastrophe), MBD_ERR_NONFINITE,
 * MBD_ERR_OOM, MBD_ERR_CUDA; outputs untouched on error.  Not reaching tol is
 * not an error: check *residual. */
mbd_status mbd_scs_screen(mbd_system *sys, int32_t n_freq, double tol, int32_t max_iter, double *alpha_out,
                          double *omega_out, double *r_vdw_out, double *c6_out, double *alpha_iu_out,
                          int32_t *iterations, double *residual);

/* ---- choice of the Ewald splitting, cutoffs and mesh (host only) ----
 * The paper's convergence study of Delta_11 against the mesh (Numerical
 * results section) finds the SPME error set by the density of mesh points,
 * independently of the system, and takes 1.2 points per angstrom along each
 * box dimension as its default.  MBD_DEFAULT_MESH_DENSITY is that density in
 * points per bohr. */
#define MBD_DEFAULT_MESH_DENSITY (1.2 / 1.8897261254578281)

/* mesh[a] = the smallest 2^a 3^b 5^c >= max(points_per_bohr x |a_a|, 2 p),
 * a_a the rows of cell (bohr).  points_per_bohr <= 0 selects
 * MBD_DEFAULT_MESH_DENSITY.  MBD_ERR_INVALID_ARG for a degenerate cell, an odd
 * or out-of-range spline order, or a mesh above 1000. */
mbd_status mbd_mesh_for_density(const double cell[9], double points_per_bohr, int32_t spline_order,
                                int32_t mesh[3]);

/* Ewald splitting beta_E, cutoffs and mesh for a target relative accuracy
 * `tol` (0 < tol < 1) of the generalized field E = T'^pbc d (relative L2
 * error over all atoms and components, for dipoles of random directions).
 * Reads desc->cell, n_atoms, r_vdw (host [N]), damp_beta, damp_d,
 * spline_order, and desc->r_cut as an upper bound on the real-space cutoff
 * (<= 0: 12 bohr); writes desc->ewald_beta, r_cut, damp_cut and mesh.  The
 * error budget is split evenly over three terms, each from an estimate that
 * was calibrated against a converged direct Ewald sum:
 *   erfc truncation    2 exp(-(beta_E r_cut)^2)
 *   damping correction 0.1 (1 - s(damp_cut)), s the Fermi damping of the
 *                      largest vdW-radius pair
 *   mesh               c_p (beta_E h)^p, h = plane spacing / K, c_4 = 0.4,
 *                      c_p = 0.1 for p >= 6
 * Cutoffs are at most 0.49 x the smallest plane spacing of the cell.
 * *est_err (may be NULL) receives the estimated error of the written
 * parameters.  Returns MBD_ERR_UNSUPPORTED (parameters still written) when the
 * cell is too small for the damping correction to reach its share of tol. */
mbd_status mbd_spme_params(mbd_system_desc *desc, double tol, double *est_err);

/* ---- batches of independent systems ----
 * The probes of one system are independent of one another, and so are whole
 * systems: the paper's parallel scheme distributes independent stochastic
 * samples with one reduction before the trace (Sections 4 and 5).  A
 * batch holds n_sys systems of uneven sizes (each its own cell, atoms and mesh)
 * on one GPU.  mbd_batch_lanczos_energy runs Algorithm 1 for every member at
 * once: the first call with a given (n_probes, n_steps) records every member's
 * whole run (probes, m Lanczos steps, quadrature, energy) as an independent
 * branch of one CUDA graph; later calls with the same (n_probes, n_steps)
 * replay that graph with new seeds.  Members cannot be reached one at a time;
 * create separate systems for that. */

/* descs: host array [n_sys] of system descriptions (each as for
 * mbd_create_system; all must share one precision).  cuda_stream: the stream
 * the batch's work is ordered on (NULL: legacy default stream); the library
 * captures on a stream of its own.  *out receives the handle on MBD_OK. */
mbd_status mbd_create_batch(int32_t n_sys, const mbd_system_desc *descs, void *cuda_stream, mbd_batch **out);

/* Release the batch, its members and its graph (NULL is ignored). */
void mbd_destroy_batch(mbd_batch *batch);

/* Energies of every member (Algorithm 1 per member).  seeds: host [n_sys],
 * member i uses seeds[i] with the probe rule of mbd_lanczos_energy, so member
 * i's energy equals mbd_lanczos_energy on the same description and seed up to
 * summation order (the kernels and their order are the same).  energies: host
 * [n_sys] (required); traces: host [n_sys] or NULL.  On a member's failure
 * (MBD_ERR_NOT_POSITIVE_DEFINITE, MBD_ERR_NONFINITE) the call returns that
 * status, writes nothing, and *failed_member (if not NULL) names the first
 * failing member. */
mbd_status mbd_batch_lanczos_energy(mbd_batch *batch, int32_t n_probes, int32_t n_steps, const uint64_t *seeds,
                                    double *energies, double *traces, int32_t *failed_member);

/* Number of members, the kernel nodes of the current graph (0 before the
 * first run) and the total atoms of the batch. */
typedef struct {
    int32_t n_sys;
    int64_t graph_kernels;
    int64_t total_atoms;
} mbd_batch_info;
mbd_status mbd_batch_get_info(const mbd_batch *batch, mbd_batch_info *info);

/* ---- storage of the Lanczos basis ----
 * The force estimator needs w_l = sum_k c_lk y_lk, which takes all m basis
 * vectors of every probe.  MBD_BASIS_STORE (the default) keeps them,
 * m x 3N x R FP64.  MBD_BASIS_RECOMPUTE keeps three and, in
 * mbd_energy_forces, reruns the recurrence after the quadrature.  The rerun uses
 * the same kernels in the same order, so it gives the same y_k, and it adds
 * c_k y_k into w as each y_k is completed.  That costs about twice the
 * Lanczos time, with memory for five vectors instead of m.  Energies are
 * identical in both modes; forces agree to rounding of the sum for w. */
enum { MBD_BASIS_STORE = 0, MBD_BASIS_RECOMPUTE = 1 };
mbd_status mbd_set_basis_storage(mbd_system *sys, int32_t mode);

/* ---- evaluation of the real-space field (Eq. fld_ewald) ----
 * MBD_REAL_PAIRS: inside the field kernel, each atom's neighbours split over
 *   the warps of a block (every neighbour's dipoles loaded once per pair).
 * MBD_REAL_CLUSTERS: a kernel of its own over clusters of 16 atoms that are
 *   consecutive in the Morton order of the mesh bricks: a warp loads each
 *   distinct neighbour (j, image) of the cluster once and applies it to every
 *   cluster atom that has it, then the field kernel adds the result.
 * MBD_REAL_AUTO (default): clusters when there are at least four per SM
 *   (and probe chunk of 64 FP32 or 32 FP64 probes), else pairs.
 * The two evaluations sum the same pairs in different orders (results agree
 * to rounding).  MBD_ERR_UNSUPPORTED for MBD_REAL_CLUSTERS when a cluster has
 * more than 4096 pairs (more than 256 neighbours per atom on average); the
 * clusters are rebuilt with every geometry. */
enum { MBD_REAL_AUTO = 0, MBD_REAL_CLUSTERS = 1, MBD_REAL_PAIRS = 2 };
mbd_status mbd_set_real_space_method(mbd_system *sys, int32_t method);

/* ---- autotuning ----
 * Times the candidate launch choices for this system at n_probes probes on the
 * system's stream and keeps the fastest.  The candidates are the FP32 FFT tile
 * width (32 or 16 complex columns), the tile width of the fused
 * spreading + first FFT pass (32 or 16), and the field kernel's atoms per
 * block (the occupancy-derived value, half and twice it, and four blocks per
 * SM).  The choices hold for later calls with the same probe width and until
 * the next mbd_autotune or mbd_set_launch_choices.  The tile widths do not
 * change any result.  The
 * atoms per block change the summation order of the a_k reductions (last-bit
 * differences).  choices (host [4], may be NULL) receives the probe width,
 * the atoms per block, the FFT tile and the spreading tile (0: not
 * applicable). */
mbd_status mbd_autotune(mbd_system *sys, int32_t n_probes, int32_t choices[4]);

/* Sets the launch choices directly, in the layout mbd_autotune returns, so
 * that a saved result can be applied again without timing.  choices[0] = 0
 * returns to the built-in rules; any other entry 0 keeps the built-in rule
 * for that choice.  MBD_ERR_INVALID_ARG for a probe width that is not even and
 * positive, atoms per block outside [0, 64], or tiles other than 0, 16 and 32
 * (0 only for an FP64 system). */
mbd_status mbd_set_launch_choices(mbd_system *sys, const int32_t choices[4]);

/* ---- stage-level entry points (per-stage checks and users of single stages) ---- */

/* The normalised probes v_l (l = first..first+R-1) of the probe rule above,
 * device FP64 [R][dim]. */
mbd_status mbd_generate_probes(uint64_t seed, int32_t first, int32_t n_probes, int32_t dim,
                               double *v_dev);

/* Generalised field E = T'^pbc d restricted to the terms in `terms`
 * (MBD_TERM_*; Eq. ewalddip): d_dev, e_dev device FP64 [nvec][N][3]. */
mbd_status mbd_field(mbd_system *sys, int32_t nvec, const double *d_dev, double *e_dev, int32_t terms);

/* SPME dipole array D(k) = sum_j d_j . grad W_j(k) (Eq. dipolarr): d_dev device
 * FP64 [nvec][N][3] -> mesh_dev device FP64 [nvec][K1][K2][K3]. */
mbd_status mbd_spread(mbd_system *sys, int32_t nvec, const double *d_dev, double *mesh_dev);

/* FFT convolution phi = F^-1[G F[D]] with the system's influence function
 * (Eq. spme): device FP64 [nvec][K1][K2][K3] in and out (may alias). */
mbd_status mbd_convolve(mbd_system *sys, int32_t nvec, const double *mesh_in_dev, double *mesh_out_dev);

/* Gauss quadrature of a batch of tridiagonals (Eqs. tridiag2, sl3): host
 * a [R][m], b [R][m] (b[l][k] couples k and k+1; the entries from the first
 * zero on are ignored), q [R] out; the default method (MBD_QUAD_CHEBYSHEV). */
mbd_status mbd_tridiag_quadrature(int32_t n_probes, int32_t n_steps, const double *a_host,
                                  const double *b_host, double *q_host);

/* The same with the method given (MBD_QUAD_*) and, if c_host is not NULL, the
 * force coefficients c = Delta^{-1/2} e_1 as host [R][m] (zeros beyond each
 * probe's length). */
mbd_status mbd_tridiag_functions(int32_t n_probes, int32_t n_steps, const double *a_host, const double *b_host,
                                 int32_t method, double *q_host, double *c_host);

/* The quadrature of mbd_tridiag_quadrature for callers that cannot let the
 * library allocate device memory: callers whose device memory belongs to
 * another allocator (a framework's caching allocator, a pool registered with a
 * communication library) or that cannot afford the device-wide
 * synchronisation that cudaMalloc and cudaFree imply.  The paper has no
 * counterpart; this is a library convenience.
 *   a_dev, b_dev  device FP64 [R][m], caller-owned, same meaning as the host
 *                 arrays of mbd_tridiag_quadrature (b[l][k] couples k and k+1;
 *                 from the first zero on, entries are ignored)
 *   q_dev         device FP64 [R] output, caller-owned
 *   cuda_stream   cudaStream_t for the work, or NULL for the legacy default stream
 * The call allocates nothing: no cudaMalloc, cudaFree or allocating library
 * routine.  Its scratch (about 2.1 MB) is one file-scope device array that every
 * GPU loading the library holds until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) and caches
 * it; make that first call before any stream capture.  The cache lives as long
 * as the process: after cudaDeviceReset on a device the cached address no
 * longer names the array, so do not call this entry point on that device
 * again in the same process.  Every call shares the
 * one array (it keeps the last call's contents; the call clears what must
 * start at zero), so calls that overlap on the GPU, for example on two streams,
 * race: serialise them.  Returns MBD_ERR_INVALID_ARG for R > MBD_NOALLOC_MAX_PROBES
 * or m > 128, MBD_ERR_NOT_POSITIVE_DEFINITE if a Ritz value is <= 0.  The call
 * returns after its work has finished. */
#define MBD_NOALLOC_MAX_PROBES 1024
mbd_status mbd_tridiag_quadrature_noalloc(int32_t n_probes, int32_t n_steps, const double *a_dev,
                                          const double *b_dev, double *q_dev, void *cuda_stream);

/* The Lanczos layer alone: the same recurrence, quadrature and estimator as
 * mbd_lanczos_energy, driven by a dense symmetric FP64 matrix C_dev [dim][dim]
 * (device).  energy = (1/2) trace - 1.5 * omega_sum. */
mbd_status mbd_lanczos_energy_dense(int32_t dim, const double *c_dev, double omega_sum,
                                    int32_t n_probes, int32_t n_steps, uint64_t seed,
                                    double *energy, double *q_host, double *ab_host);

/* Introspection: number of atoms, mesh, neighbour-pair count and the byte
 * sizes of the device arrays in use (for measurement). */
typedef struct {
    int32_t n_atoms;
    int32_t mesh[3];
    int64_t n_pairs;          /* directed real-space pairs (i, j, image) */
    int64_t device_bytes;     /* device memory held by the system */
    int32_t precision;
} mbd_info;
mbd_status mbd_get_info(const mbd_system *sys, mbd_info *info);

/* ---- tracing: per-stage launch counts and device time ---- */

/* Stages of the hot path, in the order of Algorithms 1 and 2. */
enum {
    MBD_STAGE_PROLOGUE = 0,     /* probes, y*_k, b_k (Eq. recurs2) */
    MBD_STAGE_SPREAD = 1,       /* dipole array (Eq. dipolarr) */
    MBD_STAGE_FFT = 2,          /* forward FFT, influence function, inverse FFT (Eq. spme) */
    MBD_STAGE_FIELD = 3,        /* gather + real space + self + l_k, a_k (Eqs. spme, fld_ewald, lk3) */
    MBD_STAGE_QUADRATURE = 4,   /* tridiagonal quadrature, trace, energy (Eqs. tridiag2, sl4) */
    MBD_STAGE_FORCE_PREP = 5,   /* Delta^{-1/2} e_1, w_l, (g.w_l, g.v_l) */
    MBD_STAGE_FORCE_SPREAD = 6,
    MBD_STAGE_FORCE_FFT = 7,
    MBD_STAGE_FORCE_GATHER = 8, /* Hessian gather + real-space pair gradient */
    MBD_STAGE_OTHER = 9,        /* layout transposes, setup */
    MBD_STAGE_REAL = 10,        /* real-space field of the dipoles on atom clusters (Eq. fld_ewald) */
    MBD_NUM_STAGES = 11
};

typedef struct {
    int64_t launches[MBD_NUM_STAGES];   /* kernel launches per stage since the last reset */
    double ms[MBD_NUM_STAGES];          /* device time per stage (CUDA events on the system's
                                           stream; only while timing is enabled) */
    int64_t total_launches;
} mbd_profile;

/* Reset the counters; enable = 1 also brackets every stage with CUDA events
 * on the system's stream (a few microseconds of host time per stage). */
mbd_status mbd_profile_enable(mbd_system *sys, int32_t enable);

/* Read the counters (synchronises the system's stream). */
mbd_status mbd_profile_read(mbd_system *sys, mbd_profile *out);

/* ---- failure injection (tests of the error paths; the paper has no counterpart) ----
 * The n-th device allocation of the library from now on (n = 0: the next one)
 * reports failure without calling cudaMalloc, exactly as an exhausted device
 * would: the call that needed it returns MBD_ERR_OOM with its outputs
 * untouched and the handle still usable.  One allocation fails, then the hook
 * disarms itself; n < 0 disarms it at once.  Process-wide; always MBD_OK. */
mbd_status mbd_debug_fail_allocation(int64_t n);

/* Human-readable name of a status code (static storage). */
const char *mbd_status_string(mbd_status status);

/* Last CUDA error text seen by the library in this thread ("" if none). */
const char *mbd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MBD_H */
