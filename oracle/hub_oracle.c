/*
 * hub_oracle.c -- plain, slow CPU oracle for the one-band Hubbard Hamiltonian.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline leg
 * use it.  It shares no code, header or table with the CUDA library.
 *
 * It works in the Lin-Gubernatis two-spin basis (Sec. II, Eqs. 5-6): a state is
 * the single integer I = I_up + 2^M I_dn, with site i (0-based) on bit i of I_up
 * and on bit M+i of I_dn.  The creation operators are ordered with all spin-up
 * operators (sites 1..M) left of all spin-down operators (Sec. II, Eq. 7).
 *
 * The Hamiltonian (Sec. I, Eq. 1, generalised to per-bond hopping t_b, per-site
 * interaction U_i and per-site energy eps_i):
 *     H = - sum_b t_b sum_sigma (c+_{i sigma} c_{j sigma} + h.c.)
 *         + sum_i U_i n_{i up} n_{i dn} + sum_i eps_i (n_{i up} + n_{i dn}).
 *
 * Every matrix element is produced the way Sec. III.A describes it for the
 * two-spin basis: apply a hop to the full state I, take the sign from the
 * number of same-spin electrons strictly between the two sites, and find the
 * index of the new state by binary search in the sorted list of all I
 * (Sec. V).  The diagonal counts doubly occupied sites (Sec. III.B) by a loop
 * over sites.  Nothing is blocked, fused or reordered.
 */
#include <stdint.h>
#include <stddef.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define HUBO_OK 0
#define HUBO_ERR_ARG (-1)
#define HUBO_ERR_MISSING (-2)

static int popcount64(uint64_t v) { return __builtin_popcountll(v); }

int hubo_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * All two-spin basis states of sector (n_up, n_dn) in ascending order of I
 * (Sec. II, Eqs. 5-6; the ascending order is the order of Eq. count2, with the
 * spin-up index running fastest, as Table I shows).  I_dn occupies the high M
 * bits, so scanning I_dn in the outer loop and I_up in the inner loop visits the
 * integers I in increasing order; every candidate is filtered by popcount.
 * Writes out[] when out != NULL and returns the number of states (the sector
 * dimension count_up * count_dn of Eq. count3), or a negative error.
 */
int64_t hubo_basis(int M, int n_up, int n_dn, uint64_t *out)
{
    if (M < 1 || M > 31 || n_up < 0 || n_up > M || n_dn < 0 || n_dn > M) return HUBO_ERR_ARG;
    const uint64_t lim = 1ull << M;
    int64_t k = 0;
    for (uint64_t idn = 0; idn < lim; idn++) {
        if (popcount64(idn) != n_dn) continue;
        for (uint64_t iup = 0; iup < lim; iup++) {
            if (popcount64(iup) != n_up) continue;
            if (out) out[k] = iup | (idn << M);
            k++;
        }
    }
    return k;
}

/* Index of state J in the sorted list, or -1 (binary search, Sec. V). */
static int64_t find_state(const uint64_t *basis, int64_t D, uint64_t J)
{
    int64_t lo = 0, hi = D - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        uint64_t v = basis[mid];
        if (v == J) return mid;
        if (v < J) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Diagonal element of state I: U_i per doubly occupied site plus eps_i per electron. */
static double diag_element(int M, uint64_t I, const double *U, const double *eps)
{
    double d = 0.0;
    for (int i = 0; i < M; i++) {
        int nu = (int)((I >> i) & 1u);
        int nd = (int)((I >> (M + i)) & 1u);
        d += U[i] * (double)(nu * nd) + eps[i] * (double)(nu + nd);
    }
    return d;
}

/*
 * Hop of one spin (bit offset off = 0 for up, M for down) across bond (i, j)
 * applied to the full state I.  Returns 0 when the hop is blocked (both sites
 * empty or both occupied); otherwise stores the new state and the fermion sign
 * (-1)^(number of same-spin electrons strictly between i and j), Sec. III.A, Eq. 8.
 */
static int hop(uint64_t I, int off, int i, int j, uint64_t *J, int *sign)
{
    uint64_t bi = (I >> (off + i)) & 1u, bj = (I >> (off + j)) & 1u;
    if (bi == bj) return 0;
    int lo = i < j ? i : j, hi = i < j ? j : i, between = 0;
    for (int k = lo + 1; k < hi; k++) between += (int)((I >> (off + k)) & 1u);
    *J = I ^ (1ull << (off + i)) ^ (1ull << (off + j));
    *sign = (between & 1) ? -1 : 1;
    return 1;
}

/*
 * y[n - r0] = (H x)_n for rows n in [r0, r1) (the matrix-free product of Sec. IV,
 * one output row at a time).  With absolute != 0 every matrix element and every x_m is
 * replaced by its absolute value, giving (|H| |x|)_n, the scale of per-entry tolerances.
 * bonds[2b], bonds[2b+1] are 0-based site ids.  U[M], eps[M] are per-site.  Returns 0, or HUBO_ERR_MISSING if a hopped state is
 * not in the list (which would mean the list is not a closed sector).
 */
int hubo_apply(int M, int n_bonds, const int32_t *bonds, const double *t, const double *U,
               const double *eps, const uint64_t *basis, int64_t D, const double *x, double *y,
               int64_t r0, int64_t r1, int absolute)
{
    if (r0 < 0 || r1 > D || r0 > r1) return HUBO_ERR_ARG;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 4096) reduction(| : err)
    for (int64_t n = r0; n < r1; n++) {
        uint64_t I = basis[n];
        double acc = absolute ? fabs(diag_element(M, I, U, eps) * x[n]) : diag_element(M, I, U, eps) * x[n];
        for (int b = 0; b < n_bonds; b++) {
            for (int s = 0; s < 2; s++) {
                uint64_t J;
                int sign;
                if (!hop(I, s * M, bonds[2 * b], bonds[2 * b + 1], &J, &sign)) continue;
                int64_t m = find_state(basis, D, J);
                if (m < 0) { err = 1; continue; }
                acc += absolute ? fabs(t[b] * x[m]) : -t[b] * (double)sign * x[m];
            }
        }
        y[n - r0] = acc;
    }
    return err ? HUBO_ERR_MISSING : HUBO_OK;
}

/*
 * Off-diagonal entries of row n of H: for every bond (in bond order) and spin
 * (up, then down) whose hop is allowed, the column index and value
 * -t_b * sign.  Writes at most cap entries, returns how many there are.
 */
int hubo_row(int M, int n_bonds, const int32_t *bonds, const double *t, const uint64_t *basis,
             int64_t D, int64_t n, int64_t *cols, double *vals, int cap)
{
    if (n < 0 || n >= D) return HUBO_ERR_ARG;
    uint64_t I = basis[n];
    int k = 0;
    for (int b = 0; b < n_bonds; b++) {
        for (int s = 0; s < 2; s++) {
            uint64_t J;
            int sign;
            if (!hop(I, s * M, bonds[2 * b], bonds[2 * b + 1], &J, &sign)) continue;
            int64_t m = find_state(basis, D, J);
            if (m < 0) return HUBO_ERR_MISSING;
            if (k < cap) { cols[k] = m; vals[k] = -t[b] * (double)sign; }
            k++;
        }
    }
    return k;
}

/*
 * Expectation values in a (real) state psi, read off the definition of each
 * derivative of H (Hellmann-Feynman: dE/dtheta = <psi| dH/dtheta |psi> for a
 * normalised eigenvector):
 *   dt[b]   = <psi| -sum_sigma (c+_i c_j + h.c.) |psi>   (dH/dt_b)
 *   dU[i]   = <psi| n_{i up} n_{i dn} |psi>              (dH/dU_i)
 *   deps[i] = <psi| n_{i up} + n_{i dn} |psi>            (dH/deps_i)
 * psi need not be normalised; the sums are plain quadratic forms.
 */
int hubo_expect(int M, int n_bonds, const int32_t *bonds, const uint64_t *basis, int64_t D,
                const double *psi, double *dt, double *dU, double *deps)
{
    for (int b = 0; b < n_bonds; b++) dt[b] = 0.0;
    for (int i = 0; i < M; i++) { dU[i] = 0.0; deps[i] = 0.0; }
    for (int64_t n = 0; n < D; n++) {
        uint64_t I = basis[n];
        double p2 = psi[n] * psi[n];
        for (int i = 0; i < M; i++) {
            int nu = (int)((I >> i) & 1u), nd = (int)((I >> (M + i)) & 1u);
            dU[i] += p2 * (double)(nu * nd);
            deps[i] += p2 * (double)(nu + nd);
        }
        for (int b = 0; b < n_bonds; b++) {
            for (int s = 0; s < 2; s++) {
                uint64_t J;
                int sign;
                if (!hop(I, s * M, bonds[2 * b], bonds[2 * b + 1], &J, &sign)) continue;
                int64_t m = find_state(basis, D, J);
                if (m < 0) return HUBO_ERR_MISSING;
                dt[b] += -(double)sign * psi[n] * psi[m];
            }
        }
    }
    return HUBO_OK;
}
