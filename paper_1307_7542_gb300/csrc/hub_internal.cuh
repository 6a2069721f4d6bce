// hub_internal.cuh -- handle layout, error plumbing and device helpers shared by the
// library's translation units.  Not part of the public ABI (see include/hub.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hub.h"

namespace hub {

constexpr int kMaxSites = 30;   // spin strings fit in uint32, two-spin index fits in int64
constexpr int kMaxBonds = 255;   // bond ids and per-row group lengths fit in uint8

// ---------------------------------------------------------------------------------------
// Errors: every entry point returns a code; the message goes to a thread-local string.
// ---------------------------------------------------------------------------------------
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define HUB_CUDA(call)                                                        \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) return ::hub::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define HUB_LAUNCH_CHECK() HUB_CUDA(cudaGetLastError())

// ---------------------------------------------------------------------------------------
// One-spin hopping matrix in CSR form (Sec. IV.A, Eqs. 9-10).
// ---------------------------------------------------------------------------------------
struct SpinCSR {
  int32_t *rowptr = nullptr;   // [count + 1]
  int32_t *col = nullptr;      // [nnz], ascending within a row
  double *val = nullptr;       // [nnz], -t_b * (-1)^(electrons strictly between the sites)
  uint32_t *scol = nullptr;    // [nnz], col | (sign bit << 31): -t_b = -t * sign for uniform t
  uint8_t *bond = nullptr;     // [nnz], bond id of the entry (gradients)
  int64_t nnz = 0;
  int32_t max_row = 0;
};

struct FastState;   // fast-path tables and scratch (hub_fast.cu)
struct K0State;     // k = 0 translation-sector tables (hub_k0.cu)
struct SmallState;  // single-launch Lanczos of small sectors (hub_small.cu)

// Read-only view of everything a kernel needs, passed by value.
struct Ham {
  int M;
  int64_t n_up, n_dn;                 // count_up, count_dn
  const uint32_t *basis_up, *basis_dn;
  const int32_t *rp_up, *rp_dn;       // CSR row pointers
  const int32_t *col_up, *col_dn;
  const double *val_up, *val_dn;
  const uint32_t *scol_up, *scol_dn;  // signed columns (uniform-t kernels)
  const double *eps_up, *eps_dn;      // per-state site-energy sums (nullptr when eps == 0)
  int uniform_U;                      // 1: U_i = U0 for all i
  double U0;
  double U[kMaxSites];                // per-site U_i
  int uniform_t;                      // 1: all t_b equal to t0
  double t0;
  int has_eps;
};

}  // namespace hub

// The handle behind the opaque hub_t.
struct hub_ctx {
  int device = 0;
  int M = 0;
  int N[2] = {0, 0};
  int64_t count[2] = {0, 0};
  bool shared = false;                 // N_up == N_dn: one basis and one CSR for both spins
  uint32_t *basis[2] = {nullptr, nullptr};
  uint64_t *binom = nullptr;           // device Pascal triangle, (kMaxSites+1)^2

  bool have_hop = false;
  int n_bonds = 0;
  std::vector<int32_t> bonds;
  std::vector<double> t, eps;
  hub::SpinCSR csr[2];
  double *eps_state[2] = {nullptr, nullptr};
  bool has_eps = false;

  bool have_U = false;
  bool uniform_U = true;
  double U0 = 0.0;
  std::vector<double> U;

  // Lanczos workspace (3 vectors), scalars, partial sums and the last run's coefficients.
  double *work[3] = {nullptr, nullptr, nullptr};
  double *psi_tmp = nullptr;
  double *d_scal = nullptr;            // [8] device scalars
  double *h_scal = nullptr;            // [8] pinned host mirror
  double *partials = nullptr;          // reduction partials
  int64_t partials_n = 0;
  std::vector<double> alpha, beta;

  // host-buffer apply; the second pair alternates with the first in hub_apply_host_many
  double *hx = nullptr, *hy = nullptr;
  double *hx2 = nullptr, *hy2 = nullptr;

  // |x0| of the last Lanczos run (the continued fraction of the Green's function needs it)
  double start_norm = 0.0;
  // second Lanczos pass: expand the eigenvector of T for the eigenvalue nearest psi_target
  // instead of the lowest one (hub_lanczos_ritz); psi_value records the value used
  bool psi_at_target = false;
  double psi_target = 0.0, psi_value = 0.0;
  // source index and sign per state of this handle's sector for hub_ladder
  int32_t *ladder_map = nullptr;
  int64_t ladder_cap = 0;

  // measurement: event pairs per kind (HUB_PROF_*), launch counters
  bool prof = false;
  static constexpr int kProfKinds = 4; // HUB_PROF_APPLY .. HUB_PROF_UPDATE
  std::vector<cudaEvent_t> ev_start[kProfKinds], ev_end[kProfKinds];
  int64_t n_launch[kProfKinds] = {0, 0, 0, 0};   // launches per kind since hub_profile(h, 1)
  int64_t n_timed[kProfKinds] = {0, 0, 0, 0};    // of which timed with an event pair
  int64_t n_kernels = 0;               // all kernels launched since hub_profile(h, 1)

  // fast path (double-float, two-pass apply) for uniform hopping and interaction
  hub::FastState *fast = nullptr;
  int mode = 0;                        // HUB_MODE_AUTO or HUB_MODE_FP64
  bool fail_waits = false;             // test hook: pass 1 reports a given-up wait (hub_test_fail_waits)

  // k = 0 sector of the translation i -> i-1 mod M (hub_set_symmetry); vectors are then in
  // row form, rows x cols (hub_k0.cu)
  hub::K0State *k0 = nullptr;

  // sectors of at most small_max_dim states run hub_lanczos_ground as one cooperative
  // kernel per batch of iterations (hub_small.cu); 0 turns that off
  int64_t small_max_dim = int64_t(1) << 18;
  hub::SmallState *small = nullptr;

  hub::Ham view() const;
};

namespace hub {

// Allocation helpers: on failure they set the message and return false.
bool dev_alloc(void **p, size_t bytes, const char *what);
void dev_free(void *p);
int ensure_partials(hub_ctx *h, int64_t n);

// Launch helpers.
int num_sms();
constexpr int kReduceThreads = 256;

// Deterministic FP64 reduction of partials[0..n) into *out (device), one block.
int reduce_partials(const double *partials, int n, double *out, int mode, cudaStream_t s);
// Same, in two fixed-order stages through tmp[ntmp] (for long partial lists).
int reduce_partials_2stage(const double *partials, int n, double *tmp, int ntmp, double *out, int mode,
                           cudaStream_t s);

// Apply entry used by Lanczos and the VJP (no argument checks).
int apply_launch(hub_ctx *h, const double *x, double *y, cudaStream_t s);
// The FP64 product kernel of the full sector; with a gate it does nothing unless gate[0] != 0
// when it runs (a device flag written earlier on the stream).
int f64_apply(hub_ctx *h, const double *x, double *y, const int *gate, cudaStream_t s);

// Fast path (hub_fast.cu).
bool fast_eligible(const hub_ctx *h);
int fast_build(hub_ctx *h);
void fast_release(hub_ctx *h);
int fast_apply_f64(hub_ctx *h, const double *x, double *y, cudaStream_t s);
int fast_apply_host(hub_ctx *h, const double *x_host, double *y_host, double *xd, double *yd, cudaStream_t s);
// True when the fast path's host-buffer apply runs in row chunks (staged pass 1, enough rows),
// the case fast_apply_host_many pipelines across vectors.
bool fast_host_pipelined(const hub_ctx *h);
int fast_apply_host_many(hub_ctx *h, int64_t n_vec, const double *x_host, double *y_host, double *const xd[2],
                         double *const yd[2], cudaStream_t s);
int fast_lanczos(hub_ctx *h, const double *x0, int maxit, double tol, double *E0, double *psi_out, int *iters,
                 cudaStream_t s);
int fast_check_error(hub_ctx *h);
// Lowest eigenvalues of the successive tridiagonals T_1, T_2, ... of one Lanczos run (host),
// each by bisection on the Sturm count like tridiag_lowest, but started from a bracket around
// the previous value (by Cauchy interlacing the new one lies at or below it), widened until the
// count is 0 at its lower end and at least 1 at its upper end; both bisections end on the two
// adjacent doubles where the count steps from 0 to 1, so they return the same value.
struct LowestTracker {
  double last = 0.0, step = 0.0;
  int n = 0;
  double next(const double *a, const double *b, int k);
};
double tridiag_lowest(const double *a, const double *b, int k);

// Eigenvalue of the last run's T whose eigenvector the second Lanczos pass expands (E0, or the
// one nearest h->psi_target); also stored in h->psi_value.
double psi_eigenvalue(hub_ctx *h, double E0);
inline bool use_fast(const hub_ctx *h) {
  return h->mode == HUB_MODE_AUTO && h->fast && !h->k0 && fast_eligible(h);
}

// Single-launch Lanczos of small sectors (hub_small.cu).
bool small_eligible(const hub_ctx *h);
int small_lanczos(hub_ctx *h, const double *x0, int maxit, double tol, double *E0, double *psi_out, int *iters,
                  cudaStream_t s);
int small_check_error(hub_ctx *h);
void small_release(hub_ctx *h);

// k = 0 sector (hub_k0.cu).
int64_t vec_len(const hub_ctx *h);   // length of a state vector in the handle's current layout
int k0_apply(hub_ctx *h, const double *x, double *y, cudaStream_t s);
int k0_project_inplace(hub_ctx *h, double *x, cudaStream_t s);
void k0_leave(hub_ctx *h);           // back to the full sector, vectors sized for it dropped
void k0_release(hub_ctx *h);

// Event pair around a launch of the given kind (no-op unless profiling).
int prof_mark(hub_ctx *h, int kind, bool begin, cudaStream_t s);

// Count kernel launches for the measurement hooks.
inline void count_launch(hub_ctx *h, int n = 1) {
  if (h->prof) h->n_kernels += n;
}

// Device helpers ------------------------------------------------------------------------
// Combinatorial number system (Sec. II, App. A).  binom[n * kB + k] = C(n, k);
// rank(s) = sum_j C(b_j, j) over the set bits b_1 < b_2 < ... of s (j = 1, 2, ...), the
// position of s in the ascending list of strings with its number of ones.
constexpr int kB = kMaxSites + 1;

__device__ __forceinline__ uint32_t rank_of(uint32_t s, const uint64_t *__restrict__ C) {
  uint32_t r = 0;
  int j = 1;
  while (s) {
    int b = __ffs(s) - 1;
    r += (uint32_t)C[b * kB + j];
    ++j;
    s &= s - 1;
  }
  return r;
}

// Diagonal of H at (u, d) (Sec. III.B): sum_i U_i bit_i(I_up & I_dn) + eps(I_up) + eps(I_dn).
__device__ __forceinline__ double diag_of(const Ham &H, uint32_t Iu, uint32_t Id, int64_t u, int64_t d) {
  double v;
  if (H.uniform_U) {
    v = H.U0 * (double)__popc(Iu & Id);
  } else {
    v = 0.0;
    for (uint32_t m = Iu & Id; m; m &= m - 1) v += H.U[__ffs(m) - 1];
  }
  if (H.has_eps) v += H.eps_up[u] + H.eps_dn[d];
  return v;
}

__host__ __device__ inline int popc32(uint32_t v) {
#ifdef __CUDA_ARCH__
  return __popc(v);
#else
  return __builtin_popcount(v);
#endif
}

}  // namespace hub
