/*
 * hub.h -- C ABI of the GB300 library for matrix-free Hubbard exact diagonalisation in
 * the one-spin-configuration basis (Sharma & Ahsan, "Organization of the Hilbert Space
 * for Exact Diagonalization of Hubbard Model").
 *
 * Model (Sec. I, Eq. 1, with per-bond hopping, per-site interaction and site energy):
 *     H = - sum_b t_b sum_sigma (c+_{i_b sigma} c_{j_b sigma} + h.c.)
 *         + sum_i U_i n_{i up} n_{i dn} + sum_i eps_i (n_{i up} + n_{i dn}).
 *
 * State layout (Sec. II, Eq. count2; Sec. IV.A, the vecold reshape): a vector of the
 * sector (N_up, N_dn) is the count_dn x count_up row-major matrix X, element
 * (d, u) at flat index n = d * count_up + u, where u and d are the 0-based ranks of the
 * spin strings I_up and I_dn in the ascending list of M-bit strings with N_up (N_dn)
 * bits set.  Site i (0-based) is bit i of a spin string.  With this layout
 *     H x = I_dn (x) H_up  +  H_dn (x) I_up  +  H_U            (Sec. IV.A, Eq. 11)
 * i.e. Y = X H_up^T + H_dn X + diag o X.
 *
 * Conventions for every entry point:
 *   - Return HUB_OK (0) on success, a negative HUB_ERR_* code on failure, or a positive
 *     informational code.  Nothing throws across the ABI.  hub_last_error() gives a
 *     message for the calling thread's last failure.
 *   - Pointers named *_dev are device pointers owned by the caller, pointers named
 *     *_host are host pointers owned by the caller.  Vectors are FP64, dense, of length
 *     D = count_up * count_dn, 8-byte aligned (rows * cols, the row form, while a momentum
 *     sector is active: hub_set_symmetry, hub_set_translations).
 *   - stream is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Calls that take a stream enqueue work on it and may return before it finishes,
 *     except where stated.  Set-up calls (hub_basis, hub_hopping, hub_set_U) run on
 *     the legacy default stream and return after their work is complete.
 *   - The library allocates device memory only for what a handle owns: the spin bases,
 *     the hopping matrices, per-state diagonal tables and the Lanczos workspace.  All of
 *     it is released by hub_free.
 *   - A handle is not thread-safe; calls on one handle must not overlap.
 */
#ifndef HUB_H
#define HUB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HUB_OK 0
#define HUB_CONVERGED_BREAKDOWN 1 /* Lanczos met an invariant subspace: E0 is exact there */
#define HUB_ERR_ARG (-1)          /* invalid argument (sizes, sites, bonds, NULL pointers)  */
#define HUB_ERR_OOM (-2)          /* device or host allocation failed                       */
#define HUB_ERR_CUDA (-3)         /* a CUDA runtime call failed                             */
#define HUB_ERR_NOCONV (-4)       /* Lanczos hit maxit before |dE0| < tol (E0 still set)    */
#define HUB_ERR_STATE (-5)        /* call order: e.g. hub_apply before hub_hopping           */
#define HUB_ERR_TIMEOUT (-6)      /* a device-side bounded wait gave up                      */

#define HUB_SPIN_UP 0
#define HUB_SPIN_DN 1

#define HUB_MODE_AUTO 0   /* fast double-float path when t and U are uniform (window and
                             bound: see hub_apply), else FP64; in a momentum sector:
                             integer-pipe sums when t is uniform                         */
#define HUB_MODE_FP64 1   /* always the native FP64 kernels                              */

#define HUB_SYM_NONE 0    /* the full sector (N_up, N_dn)                              */
#define HUB_SYM_K0 1      /* its k = 0 subspace under the translation i -> i-1 mod M   */
#define HUB_SYM_KPI 2     /* its k = pi subspace (T eigenvalue -1; M even)             */

#define HUB_PROF_APPLY 0  /* a whole product H x (both passes on the fast path)       */
#define HUB_PROF_UP 1     /* fast path pass 1: spin-up hops + diagonal                 */
#define HUB_PROF_DN 2     /* fast path pass 2: spin-down hops + epilogue               */
#define HUB_PROF_UPDATE 3 /* fast Lanczos: the update r_j = w - c r_{j-1} (its own pass) */

typedef struct hub_ctx *hub_t;

/* Message for the calling thread's most recent failure ("" if none). */
const char *hub_last_error(void);

/*
 * Sector set-up: counts and one-spin bases (Sec. II, Eqs. count2-count3, Appendix A).
 * M sites (1 <= M <= 30), n_up, n_dn electrons (0 <= n <= M).  Builds on the GPU the
 * ascending lists of M-bit strings with n_up and n_dn bits set (Algorithm I's order),
 * by combinadic unranking; when n_up == n_dn the two spins share one list (Sec. X).
 * On success *out owns the handle; release it with hub_free.
 */
int hub_basis(int M, int n_up, int n_dn, hub_t *out);

/* count_up = C(M, n_up) and count_dn = C(M, n_dn) (Eq. count3); either pointer may be NULL. */
int hub_dims(hub_t h, int64_t *n_up, int64_t *n_dn);

/* Copy the spin basis (uint32 strings, ascending) of spin 0 (up) or 1 (down) to host. */
int hub_get_basis(hub_t h, int spin, uint32_t *basis_host);

/*
 * One-spin hopping matrices H_up and H_dn (Sec. III.A, Eq. 8; Sec. IV.A, Eqs. 9-10),
 * built on the GPU in CSR form.  bonds_host[2b], bonds_host[2b+1] are the 0-based sites
 * of undirected bond b (b < n_bonds <= 255), i != j, no bond listed twice; t_host[b] its
 * hopping.  eps_host[M] are site energies or NULL for zero.  For a spin string s and a
 * bond (i, j) with exactly one end occupied the row of s holds the column
 * rank(s ^ (1<<i) ^ (1<<j)) with value -t_b * (-1)^(popcount of s strictly between i
 * and j); columns are ascending within a row.  May be called again to change t / eps.
 */
int hub_hopping(hub_t h, int n_bonds, const int32_t *bonds_host, const double *t_host,
                const double *eps_host);

/* On-site interaction: n_U == 1 for a uniform U, or n_U == M for per-site U_i. */
int hub_set_U(hub_t h, int n_U, const double *U_host);

/* Shape of a spin's CSR: number of nonzeros and longest row.  Either pointer may be NULL. */
int hub_csr_info(hub_t h, int spin, int64_t *nnz, int32_t *max_row);

/* Copy a spin's CSR to host: rowptr[count+1], cols[nnz] (int32), vals[nnz] (FP64). */
int hub_get_csr(hub_t h, int spin, int32_t *rowptr_host, int32_t *cols_host, double *vals_host);

/*
 * y = H x (Sec. IV.A, Eq. 11, applied matrix-free as X H_up^T + H_dn X + diag o X;
 * Sec. III.B for the diagonal, evaluated from popcount(I_up & I_dn) on the fly).
 * x_dev and y_dev must not overlap.  Requires hub_hopping and hub_set_U.
 *
 * Accuracy: every entry satisfies |y_n - (Hx)_n| <= 1e-13 (|H||x|)_n, |H| the entrywise
 * absolute matrix.  The native FP64 kernel (HUB_MODE_FP64; non-uniform t or U) does
 * this with FP64 multiply-adds.  In HUB_MODE_AUTO with uniform t and U the product runs
 * in double-float arithmetic (pairs of FP32 numbers, 48 significant bits; compensated
 * sums) with a derived worst-case error of max(N + 10.1, 16) * 2^-48 (|H||x|)_n, N <= 15 the
 * most terms one low-part accumulator takes (N = 9 on the 4x4 lattice: 6.8e-14 (|H||x|)_n).
 * That bound needs a window, checked on the device for every call: the largest |x_n| in
 * [2^-823, 2^877], every nonzero |x_n| at least 2^-80 times the largest (no FP64
 * subnormals, infinities or NaN); and a model with uniform t != 0 and U, no site energies,
 * |t| and U/|t| either 0 or in [2^-16, 2^16].  A vector or model outside it is multiplied by the FP64 kernel
 * instead, on the same stream and with no host synchronisation, so every call meets the
 * bound.
 */
int hub_apply(hub_t h, const double *x_dev, double *y_dev, void *stream);

/*
 * The same product on host buffers: copies x_host to the device, applies H, copies the
 * result to y_host, and returns when y_host is complete.  Uses two device vectors the
 * handle allocates on first use.  Accuracy, window and routing as for hub_apply.
 */
int hub_apply_host(hub_t h, const double *x_host, double *y_host, void *stream);

/*
 * y_v = H x_v for n_vec host vectors (Sec. IV.A, Eq. 11, as hub_apply): x_host holds the
 * vectors one after another (n_vec * D doubles, D the sector's vector length), y_host receives
 * the results in the same layout; returns when all of y_host is complete.  x_host and y_host
 * are either the same array (the product in place) or do not overlap at all; page-locked
 * buffers let the copies run at the link's rate.  Each result is bit for bit that of
 * hub_apply_host on the same vector (same kernels, window check and routing).  On the fast
 * path with row-chunked copies (pass 1 staging rows, at least 16 rows) the copies of
 * neighbouring vectors overlap: vector v + 1 comes in and vector v - 1 goes back while vector
 * v is computed, on two copy streams of the handle; this takes a second pair of device
 * vectors (2 D doubles more), allocated on first use.  Elsewhere it is one hub_apply_host
 * per vector.
 *   - n_vec = 0: nothing happens.  n_vec < 0, a NULL vector with n_vec > 0, partly
 *     overlapping arrays, or n_vec * D * 8 bytes beyond size_t: HUB_ERR_ARG.
 */
int hub_apply_host_many(hub_t h, int64_t n_vec, const double *x_host, double *y_host, void *stream);

/*
 * Ground state by plain Lanczos without re-orthogonalisation (Sec. IV; Sec. V).
 * q_1 = x0/|x0| (x0_dev == NULL: a uniform [-1, 1) vector from SplitMix64, seed 0).
 * Each iteration: w = H q_j - beta_{j-1} q_{j-1}; alpha_j = <q_j, w>; w -= alpha_j q_j;
 * beta_j = |w|; E0_j = lowest eigenvalue of the tridiagonal T_j.  Stops when
 * |E0_j - E0_{j-1}| < tol (tol <= 0: run exactly maxit iterations), on breakdown
 * (beta_j <= 1e-14 |alpha_j|, returns HUB_CONVERGED_BREAKDOWN) or at maxit (returns
 * HUB_ERR_NOCONV, *E0 still set).  If psi_dev != NULL the recurrence is run a second
 * time to form the normalised ground-state vector.  Blocks until done; *E0 and *iters
 * are host pointers (iters may be NULL).  Workspace: three device vectors.
 * In HUB_MODE_AUTO with uniform t and U (and t, U, eps in hub_apply's parameter range)
 * the Lanczos vectors are held in double-float form: x0 is scaled by a power of two so
 * that its largest entry lies in [1, 2), and components smaller than about 2^-126 times
 * the largest entry of a Lanczos vector are flushed.  Neither changes E0 at the 1e-10
 * level; HUB_MODE_FP64 keeps every vector in FP64.  Sectors of at most hub_set_small_dim's
 * bound (default 262144 states; not in a momentum sector) run instead in one cooperative
 * kernel per batch of iterations, FP64 throughout, in either mode: the same recurrence and
 * stopping rule, alpha_j and beta_j equal to the other drivers' up to rounding.
 */
int hub_lanczos_ground(hub_t h, const double *x0_dev, int maxit, double tol, double *E0,
                       double *psi_dev, int *iters, void *stream);

/* The alpha_j, beta_j of the last hub_lanczos_ground (host arrays of length >= cap; *n =
 * number of steps).  beta_{n-1} is 0 when the run stopped before computing it. */
int hub_lanczos_coeffs(hub_t h, double *alpha_host, double *beta_host, int cap, int *n);

/*
 * The ground state and a few low-lying excited states (Sec. IV: Lanczos for "the ground
 * state and a few low-lying excited states"): maxit steps of the plain recurrence of
 * hub_lanczos_ground from x0_dev (NULL: the seeded uniform start vector), then the
 * eigenvalues of the tridiagonal T (bisection on Sturm counts).  Without
 * re-orthogonalisation T acquires spurious copies of converged eigenvalues; they are removed
 * by the Cullum-Willoughby test: numerically multiple eigenvalues of T are kept once, and a
 * simple eigenvalue is discarded when T without its first row and column has it too
 * (tolerance 1e-10 max(1, |T|)).  Returns the lowest n_found <= n_eig distinct values in
 * eig_host (ascending) and, if resid_host != NULL, the residual estimate
 * |beta_{k-1} s_{k-1}| of each (s the normalised eigenvector of T): values whose estimate
 * is not small have not converged.  A single start vector resolves each eigenvalue once,
 * whatever its multiplicity.  1 <= maxit <= 3000 (the host eigenvalue step is O(maxit^2));
 * blocks until done; host outputs.
 */
int hub_lanczos_spectrum(hub_t h, const double *x0_dev, int maxit, int n_eig, double *eig_host, double *resid_host,
                         int *n_found, void *stream);

/*
 * Low-lying levels with their multiplicities by block Lanczos (Sec. IV's recurrence on a block
 * of k start vectors; a single start vector finds each degenerate level once).  X0_dev: k
 * vectors of the handle's vector length, contiguous (vector c at c * length), linearly
 * independent; NULL: SplitMix64 uniform [-1, 1) vectors (counter offset c * length, so the
 * first equals hub_lanczos_ground's default).  steps block steps of
 *   W = H Q_j - Q_{j-1} B_{j-1}^T, A_j = Q_j^T W, W -= Q_j A_j, full re-orthogonalisation
 *   against all earlier blocks (twice), Q_{j+1} B_j = W (Cholesky QR, twice),
 * then the eigenvalues of the block-tridiagonal matrix of the A_j and B_j (dense, on the host):
 * the lowest min(n_eig, k * steps) into eig_host, ascending, a level of multiplicity g <= k
 * appearing g times, and, if resid_host != NULL, the residual norms |H y - theta y| of their
 * Ritz vectors (|B_m s_m|; 0 when the space became invariant, which ends the steps early).
 * 1 <= k <= 8, k * steps <= 512.  Device memory: (steps + 2) * k vectors, allocated and freed
 * by the call.  Products as hub_apply (fast or FP64 path); works inside a momentum sector.
 * Blocks until done; *n_found = number of values written.
 */
int hub_lanczos_block(hub_t h, int k, const double *X0_dev, int steps, int n_eig, double *eig_host,
                      double *resid_host, int *n_found, void *stream);

/*
 * Eigenvector of a low-lying excited state (Sec. IV): maxit steps of the plain recurrence
 * from x0_dev (NULL: the seeded start vector), then the second pass of hub_lanczos_ground
 * forms the normalised Ritz vector psi_dev (device, count_up * count_dn) for the eigenvalue
 * of T nearest `target` (e.g. one returned by hub_lanczos_spectrum with the same x0 and
 * maxit); *ritz_host receives that eigenvalue.  1 <= maxit <= 3000; blocks until done.
 */
int hub_lanczos_ritz(hub_t h, const double *x0_dev, int maxit, double target, double *psi_dev, double *ritz_host,
                     void *stream);

/*
 * One-particle Green's function at zero temperature (Sec. VII, Eq. count8):
 *   G_s(p, z) = <psi0| c_ps (z + E0 - H)^-1 c+_ps |psi0> + <psi0| c+_ps (z - E0 + H)^-1 c_ps |psi0>,
 * each term a continued fraction from the Lanczos recurrence started at c+_ps psi0 or
 * c_ps psi0.  Three calls: hub_ladder forms the start vector, hub_green_coeffs runs the
 * recurrence, hub_green_eval sums the continued fraction.
 *
 * hub_ladder: y = c+_{site,spin} x (create != 0) or c_{site,spin} x (create == 0), the vecin
 * construction of Sec. VII.  x (device, length count_up * count_dn of `from`) is a vector of
 * the sector of `from`; y (device, length of `to`) is written in the sector of `to`, which
 * must have the same M, one more (create) or one fewer electron of the given spin and the
 * same number of the other spin.  Layout of hub_apply (n = d * count_up + u).  The sign is
 * the Jordan-Wigner sign of the operator order of Sec. II, Eq. 7 (all up operators before
 * all down operators, ascending sites): (-1)^(electrons of the same spin on sites below
 * `site`), times (-1)^N_up for a down-spin operator.  Entries of y whose state has no
 * preimage are 0.  Every entry of y is +-1 times one entry of x or 0, so the result is exact.
 * site in [0, M), spin HUB_SPIN_UP / HUB_SPIN_DN; x and y must not overlap.  The handles need
 * only their bases (hub_basis); `to` keeps a map of count_{spin} ints of `to`.  Asynchronous
 * on `stream`.  HUB_ERR_ARG on bad arguments or mismatched sectors.
 */
int hub_ladder(hub_t from, hub_t to, int site, int spin, int create, const double *x_dev, double *y_dev,
               void *stream);

/*
 * Continued-fraction coefficients: k steps of the plain Lanczos recurrence of
 * hub_lanczos_ground on handle h started from v (device, unnormalised, e.g. from
 * hub_ladder).  Host outputs: alpha_host[k], beta_host[k] (alpha_j, beta_j as in
 * hub_lanczos_coeffs; fewer than k when the Krylov space is exhausted, beta of the last
 * step is then ~0), *norm2_host = |v|^2 and *k_out = steps done (0 with |v| = 0).  Blocks
 * until done.  Uses h's Lanczos workspace.
 */
int hub_green_coeffs(hub_t h, const double *v_dev, int k, double *alpha_host, double *beta_host,
                     double *norm2_host, int *k_out, void *stream);

/*
 * G(z) = norm2 / (z - s (alpha_0 - E0) - beta_0^2 / (z - s (alpha_1 - E0) - ... -
 *        beta_{k-2}^2 / (z - s (alpha_{k-1} - E0))))
 * at n_z complex points z = z_re[i] + i z_im[i]; s = +1 for the particle term (coefficients
 * of c+ psi0 in sector N + 1), s = -1 for the hole term (c psi0 in sector N - 1) of
 * Eq. count8.  Host arrays only, no GPU work; G = 0 when k = 0.  HUB_ERR_ARG on bad
 * arguments.
 */
int hub_green_eval(int k, const double *alpha, const double *beta, double norm2, double E0, int sign, int n_z,
                   const double *z_re, const double *z_im, double *g_re, double *g_im);

/*
 * Many small ground states in one persistent kernel launch (Sec. VIII: an impurity solver
 * repeats the ground-state search for every sector and bath-parameter set).  One lattice
 * (1 <= M <= 16 sites, n_bonds bonds as in hub_hopping), n_params parameter sets
 * t_host[n_params][n_bonds], U_host[n_params][M], eps_host[n_params][M] (or NULL), and
 * n_jobs jobs: job k finds the lowest eigenvalue of sector (job_nup[k], job_ndn[k]) with
 * parameter set job_param[k] by the plain Lanczos of hub_lanczos_ground (FP64; E0_j of T_j
 * is checked every 8 iterations, stop when it changes by less than tol between checks;
 * start vector SplitMix64 uniform [-1, 1) with counter (k << 32) | (element + 1)).  Each
 * job's vectors live in shared memory: count_up * count_dn <= 8192 per job, else
 * HUB_ERR_ARG.  Host outputs E0_host[n_jobs], iters_host[n_jobs], status_host[n_jobs]
 * (HUB_OK, HUB_CONVERGED_BREAKDOWN or HUB_ERR_NOCONV per job).  Returns HUB_ERR_NOCONV if any
 * job hit maxit (1 <= maxit <= 1000).  Allocates and frees its own device copies; blocks.
 */
int hub_batch_ground(int M, int n_bonds, const int32_t *bonds_host, int n_params, const double *t_host,
                     const double *U_host, const double *eps_host, int n_jobs, const int32_t *job_nup,
                     const int32_t *job_ndn, const int32_t *job_param, int maxit, double tol,
                     double *E0_host, int32_t *iters_host, int32_t *status_host, void *stream);

/*
 * Hellmann-Feynman gradients of E0 = <psi|H|psi> for a normalised eigenvector psi:
 *   dE_dt[b]   = <psi| -sum_sigma (c+_i c_j + h.c.) |psi>     (dH/dt_b, per bond)
 *   dE_dU[i]   = <psi| n_{i up} n_{i dn} |psi>                (double occupancy, per site)
 *   dE_deps[i] = <psi| n_{i up} + n_{i dn} |psi>              (density, per site)
 * Host outputs (n_bonds, M, M doubles); any may be NULL.  Blocks until done.
 * For an unnormalised psi the results are the quadratic forms psi^T (dH/dtheta) psi.
 */
int hub_grad(hub_t h, const double *psi_dev, double *dE_dt_host, double *dE_dU_host,
             double *dE_deps_host, void *stream);

/*
 * hub_grad without any memory allocation (the paper has no counterpart; this is a service
 * for callers).  Some callers cannot allocate device memory at call time: code that
 * owns the whole device through its own memory pool (the pool would have to give memory
 * back), code on a latency-critical path (cudaMalloc and cudaFree can synchronise the
 * device), and code that must not change the device's memory footprint after start-up.
 * This entry point computes the same quadratic forms as hub_grad, but its scratch (per-
 * block partial sums and the reduced results) is a fixed array of 779,520 bytes compiled
 * into the library, which every GPU that loads the library holds until the process exits.
 * The caller still owns psi and the host output arrays; the handle's own tables were
 * allocated when it was built.
 *   - Limit: n_bonds + 2*M <= 160; larger models return HUB_ERR_ARG (use hub_grad).
 *   - The handle's device must be the current device.  Every call looks up the array's
 *     device address there (cudaGetSymbolAddress); the first call on a device may also
 *     load the library's device code on it, which places the array.
 *   - All calls share the one array: calls that overlap on the GPU (two streams, two
 *     threads, two handles) race and give wrong results.  Every value a call reads from
 *     the array is written earlier in the same call, so nothing needs clearing.
 *   - Blocks: every call synchronises its stream and returns after the results are in the
 *     host arrays.
 */
int hub_grad_noalloc(hub_t h, const double *psi_dev, double *dE_dt_host, double *dE_dU_host,
                     double *dE_deps_host, void *stream);

/*
 * Vector-Jacobian product of y = H(theta) x for a cotangent ybar:
 *   xbar_dev = H ybar (H is symmetric), and the parameter cotangents
 *   tbar[b] = ybar^T (dH/dt_b) x, Ubar[i] = ybar^T (dH/dU_i) x, epsbar[i] = ybar^T (dH/deps_i) x
 * (host outputs; any of the four outputs may be NULL).  Blocks until done.
 */
int hub_apply_vjp(hub_t h, const double *ybar_dev, const double *x_dev, double *xbar_dev,
                  double *tbar_host, double *Ubar_host, double *epsbar_host, void *stream);

/*
 * Translation symmetry (Sec. V): restrict the handle to the k = 0 subspace of the
 * translation T c+_{i sigma} T^-1 = c+_{i-1 sigma} (site 0 -> site M-1; the direction of the
 * paper's Tables I and II), about M times smaller than the sector.  HUB_SYM_KPI selects the
 * k = pi subspace instead (T Psi = -Psi; an extension beyond the paper's k = 0, the other
 * momentum whose Bloch states are real; M must be even, else HUB_ERR_ARG).  Everything
 * below holds for both, with "k = 0" read as the selected momentum.
 *   - Requires hub_hopping and hub_set_U first, a bond set that T maps onto itself with equal
 *     t (a ring, a ring with further-neighbour bonds, ...), uniform U and uniform eps;
 *     otherwise HUB_ERR_ARG.  HUB_ERR_OOM if one k = 0 vector would not fit on the device.
 *   - Layout ("row form", the order of the paper's Table I): the strings of each spin are
 *     grouped into T-cycles; the smallest member of a cycle is its representative.  Rows:
 *     the up representatives R_i (i = 0 .. rows-1, ascending; hub_k_reps gives them and
 *     their periods P_i).  Columns: the down representatives R_j ascending, each followed by
 *     its translations, column c = (j, n) for n = 0 .. P_j - 1 (hub_k_columns gives the
 *     string d_c of T^n R_j and the sign s_c with T^n |R_j> = s_c |d_c>); cols = count_dn.
 *     A state Psi of the sector is stored as the rows x cols FP64 array
 *         X[i * cols + c] = sqrt(P_i) * s_c * Psi(R_i, d_c),
 *     and the plain dot product of two such arrays is the inner product of the states.
 *     Rows with P_i < M hold tied entries (a cycle of T^P_i within each column block);
 *     hub_k_project enforces the ties, and entries of cycles with no state in the sector are
 *     zero.  dim (hub_k_dims) is the number of independent entries, the dimension of the
 *     sector.
 *   - While it is active, vectors of hub_apply, hub_apply_host, hub_lanczos_ground,
 *     hub_lanczos_spectrum, hub_lanczos_ritz and hub_green_coeffs are row-form arrays of
 *     length rows * cols; start vectors are projected; products always return projected
 *     arrays.  hub_grad, hub_grad_noalloc, hub_apply_vjp and hub_ladder return
 *     HUB_ERR_STATE.  hub_hopping and hub_set_U return the handle to the full sector.
 *   - Changing the symmetry frees the handle's Lanczos workspace (it is sized per layout).
 *   - Blocks until the tables are built.  HUB_SYM_NONE returns to the full sector.
 */
int hub_set_symmetry(hub_t h, int sym);

/*
 * Several commuting translations (a torus and the like): restrict the handle to the sector
 * g Psi = chi(g) Psi of the abelian group G generated by n_gen site permutations (perm_host,
 * n_gen x M: generator a moves site i to perm_host[a * M + i]) with real character values
 * char_host[a] = +1 or -1 on the generators (k = 0 or pi along each).  Sec. V's construction
 * with G in place of the powers of T; hub_set_symmetry(h, HUB_SYM_K0 / HUB_SYM_KPI) is the
 * case n_gen = 1, perm = (i -> i-1 mod M).
 *   - HUB_ERR_ARG unless: every generator is a permutation of the sites that maps the bonds
 *     onto bonds with equal t; the generators commute; G has at most 64 elements; the
 *     values define a character (-1 on a generator of odd order does not); U and eps are
 *     uniform.  1 <= n_gen <= 8.
 *   - Layout and everything else as for hub_set_symmetry, with orbits of G in place of
 *     T-cycles: rows the up representatives (smallest member of each orbit) with their orbit
 *     sizes P_i (hub_k_reps), columns each down representative followed by its images under
 *     the coset representatives of its stabiliser (the smallest element of each coset, the
 *     elements numbered breadth-first from the identity over the generators in order;
 *     hub_k_columns), X[i * cols + c] = sqrt(P_i) * s_c * Psi(R_i, d_c).
 */
int hub_set_translations(hub_t h, int n_gen, const int32_t *perm_host, const int32_t *char_host);

/* Row-form shape and dimension of the momentum sector.  HUB_ERR_STATE outside one. */
int hub_k_dims(hub_t h, int64_t *rows, int64_t *cols, int64_t *dim);

/* Up representatives R_i and periods P_i of the rows (host arrays of length rows). */
int hub_k_reps(hub_t h, uint32_t *rep_host, int32_t *period_host);

/* Down string d_c and sign s_c of every column (host arrays of length cols). */
int hub_k_columns(hub_t h, uint32_t *dn_host, int32_t *sign_host);

/*
 * y_dev = the row-form array x_dev with the ties of the short rows enforced (the
 * orthogonal projection onto the k = 0 space in row form); x_dev == y_dev is allowed,
 * other overlaps are HUB_ERR_ARG.  Enqueued on stream.
 */
int hub_k_project(hub_t h, const double *x_dev, double *y_dev, void *stream);

/*
 * Arithmetic path (no counterpart in the paper).  HUB_MODE_AUTO (default) runs products
 * with uniform t and U on the fast path: vectors held as pairs of FP32 numbers (about 48
 * significant bits), sums by error-free transformations on the FP32 pipe, because the
 * FP64 unit of this GPU issues about 1/70 of the FP32 rate.  Its per-entry error is at
 * most 6.8e-14 (|H||x|)_n at 4x4 inside the window stated at hub_apply, and inputs outside
 * the window go to the FP64 kernel, so both modes meet 1e-13 (|H||x|)_n.  Inputs and
 * outputs of every entry point stay FP64.  HUB_MODE_FP64 forces the native FP64 kernels.
 */
int hub_set_mode(hub_t h, int mode);

/*
 * Small-sector Lanczos (no counterpart in the paper): hub_lanczos_ground (and the calls built
 * on it: spectra, Ritz vectors, Green's-function coefficients) runs sectors of at most max_dim
 * states as one kernel per batch of iterations whose CTAs meet at barriers between the phases
 * of an iteration: up to 8192 states one thread-block cluster (hardware cluster barriers),
 * above that a cooperative grid (bounded waits: a wait that gives up sets the handle's error
 * flag and hub_lanczos_ground returns HUB_ERR_TIMEOUT).  This removes the per-iteration
 * launches and host round trips that bound small sectors.  max_dim = 0 turns it off; the
 * default is 262144.  HUB_ERR_ARG for a NULL handle or max_dim < 0.
 */
int hub_set_small_dim(hub_t h, int64_t max_dim);

/*
 * Waits for the handle's queued work and reports a device-side failure: HUB_ERR_TIMEOUT
 * if a bounded wait inside a kernel gave up since the last check (the flag is cleared),
 * HUB_ERR_CUDA on a CUDA error, else HUB_OK.  hub_lanczos_ground checks this itself.
 */
int hub_check(hub_t h);

/*
 * Test hook (no counterpart in the paper; off by default).  While enabled, every CTA of the
 * fast path's first pass, once the bulk copies of its first row pair have landed, and every
 * CTA of the small-sector Lanczos, before its first grid barrier, takes the exit a given-up
 * bounded wait takes: it sets the handle's device error flag and returns without computing.  No wait runs out and no copy is left in flight; the hook exists so
 * that the error path (hub_check and hub_lanczos_ground returning HUB_ERR_TIMEOUT) can be
 * exercised.  Results computed while it is enabled are meaningless.
 */
int hub_test_fail_waits(hub_t h, int enable);

/*
 * Measurement hooks (no counterpart in the paper).  hub_profile(h, 1) resets the counters
 * and starts recording a CUDA event pair on the launching stream around every product
 * (HUB_PROF_APPLY), every fast-path pass (HUB_PROF_UP, HUB_PROF_DN) and every separate
 * Lanczos update pass of the fast driver (HUB_PROF_UPDATE); up to 65536 launches per kind are
 * timed, later ones only counted.  hub_profile(h, 0) stops.
 * hub_profile_read waits for the events and returns, for one kind, the summed time in
 * milliseconds and the number of launches, plus the number of kernels the handle launched
 * since profiling started.  Any output pointer may be NULL.
 */
int hub_profile(hub_t h, int enable);
int hub_profile_read(hub_t h, int kind, double *ms, int64_t *launches, int64_t *kernel_launches);

/* Release a handle and everything it owns.  NULL is ignored. */
void hub_free(hub_t h);

#ifdef __cplusplus
}
#endif

#endif /* HUB_H */
