// hub_lanczos.cu -- plain Lanczos ground state (K4) on top of the matrix-free apply.
//
// Sec. IV: only the product H q is needed to span the Krylov space K_j(H, q); Sec. V: the
// simplest Lanczos without re-orthogonalisation gives the ground state of Table IV.  Each
// iteration here:  w = H q_j;  w -= beta_{j-1} q_{j-1};  alpha_j = <q_j, w>;
// w -= alpha_j q_j;  beta_j = |w|;  q_{j+1} = w / beta_j.  The FP64 dot products are
// reduced per block with warp shuffles, then across blocks in a fixed order, so results
// do not depend on scheduling.  E0_j, the lowest eigenvalue of the tridiagonal T_j, is
// found on the host by Sturm-sequence bisection; the ground-state vector comes from a
// second pass with the eigenvector of T (inverse iteration).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hub_internal.cuh"

namespace hub {

int ready(const hub_ctx *h, const char *who);

constexpr int kVecThreads = 256;

static int vec_grid() { return num_sms() * 4; }

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum into partials[blockIdx.x] (fixed order within the block).
__device__ __forceinline__ void block_partial(double v, double *partials) {
  __shared__ double ws[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) ws[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double s = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) partials[blockIdx.x] = s;
  }
}

// partials <- sum_k a_k b_k
__global__ void k_dot(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
                      double *__restrict__ partials) {
  double v = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    v = fma(a[k], b[k], v);
  block_partial(v, partials);
}

// w -= (*beta_prev) q_prev;  partials <- <q, w>
__global__ void k_sub_dot(int64_t n, double *__restrict__ w, const double *__restrict__ q_prev,
                          const double *__restrict__ q, const double *__restrict__ beta_prev,
                          double *__restrict__ partials) {
  const double bp = *beta_prev;
  double v = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double wk = fma(-bp, q_prev[k], w[k]);
    w[k] = wk;
    v = fma(q[k], wk, v);
  }
  block_partial(v, partials);
}

// w -= (*alpha) q;  partials <- |w|^2
__global__ void k_sub_norm(int64_t n, double *__restrict__ w, const double *__restrict__ q,
                           const double *__restrict__ alpha, double *__restrict__ partials) {
  const double a = *alpha;
  double v = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double wk = fma(-a, q[k], w[k]);
    w[k] = wk;
    v = fma(wk, wk, v);
  }
  block_partial(v, partials);
}

// w /= *beta; the first thread also records beta as the next beta_prev.
__global__ void k_scale_inv(int64_t n, double *__restrict__ w, double *__restrict__ scal) {
  const double inv = 1.0 / scal[1];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    w[k] *= inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) scal[2] = scal[1];
}

// dst = src / *nrm
__global__ void k_copy_scaled(int64_t n, double *__restrict__ dst, const double *__restrict__ src,
                              const double *__restrict__ nrm) {
  const double inv = 1.0 / *nrm;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = src[k] * inv;
}

// v /= *nrm (in place)
__global__ void k_scale_by(int64_t n, double *__restrict__ v, const double *__restrict__ nrm) {
  const double inv = 1.0 / *nrm;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    v[k] *= inv;
}

// y += a x
__global__ void k_axpy(int64_t n, double a, const double *__restrict__ x, double *__restrict__ y) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    y[k] = fma(a, x[k], y[k]);
}

// w = H q already in w:  w -= a q + b q_prev;  then w /= c  (second pass, known coefficients)
__global__ void k_recur(int64_t n, double *__restrict__ w, const double *__restrict__ q,
                        const double *__restrict__ q_prev, double a, double b, double inv_c) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    w[k] = (w[k] - a * q[k] - b * q_prev[k]) * inv_c;
}

// Start vector for x0 == NULL: uniform [-1, 1) from SplitMix64 (seed 0, counter k).
__global__ void k_splitmix_uniform(int64_t n, double *__restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = (uint64_t)(k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    out[k] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

// ---------------------------------------------------------------------------------------
// Host: symmetric tridiagonal T (diag a[0..k), off-diagonal b[0..k-1)).
// ---------------------------------------------------------------------------------------

// Number of eigenvalues of T smaller than x (Sturm sequence of the LDL^T pivots).
static int sturm_count(const double *a, const double *b, int k, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < k; ++i) {
    double bb = i ? b[i - 1] * b[i - 1] : 0.0;
    d = (a[i] - x) - (i ? bb / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

// Bisection of [lo, hi] (count 0 at lo, >= 1 at hi) down to adjacent doubles.
static double bisect_lowest(const double *a, const double *b, int k, double lo, double hi) {
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(a, b, k, mid) >= 1) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

double tridiag_lowest(const double *a, const double *b, int k) {
  if (k == 1) return a[0];
  double lo = INFINITY, hi = -INFINITY;
  for (int i = 0; i < k; ++i) {
    double r = (i ? fabs(b[i - 1]) : 0.0) + (i < k - 1 ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  return bisect_lowest(a, b, k, lo, hi);
}

double LowestTracker::next(const double *a, const double *b, int k) {
  double e;
  if (n < 2 || k == 1 || !std::isfinite(last) || !std::isfinite(step)) {
    e = tridiag_lowest(a, b, k);
  } else {
    double d = fmax(2.0 * step, 4e-16 * fmax(1.0, fabs(last)));
    double lo = last - d, hi = last + d;
    bool ok = true;
    for (int t = 0; ok && sturm_count(a, b, k, hi) < 1; ++t) {
      hi += d;
      d *= 4.0;
      ok = t < 40;
    }
    for (int t = 0; ok && sturm_count(a, b, k, lo) >= 1; ++t) {
      lo -= d;
      d *= 4.0;
      ok = t < 40;
    }
    e = ok ? bisect_lowest(a, b, k, lo, hi) : tridiag_lowest(a, b, k);
  }
  if (n > 0) step = fabs(e - last);
  last = e;
  ++n;
  return e;
}

// Eigenvector of T for eigenvalue lam by inverse iteration (tridiagonal LU with partial
// pivoting), normalised, first nonzero component positive.
std::vector<double> tridiag_vector(const double *a, const double *b, int k, double lam) {
  std::vector<double> v(k, 1.0);
  if (k == 1) return v;
  const double scale = fabs(lam) + 1.0;
  const double shift = lam - 1e-13 * scale;   // keep T - shift*I nonsingular
  // U has three diagonals u0, u1, u2; L multipliers m and pivot flags
  std::vector<double> u0(k), u1(k), u2(k), m(k), dl(k), dd(k), du(k);
  std::vector<char> piv(k, 0);
  for (int i = 0; i < k; ++i) {
    dd[i] = a[i] - shift;
    du[i] = i < k - 1 ? b[i] : 0.0;
    dl[i] = i < k - 1 ? b[i] : 0.0;   // sub-diagonal entry (i+1, i)
  }
  // Gaussian elimination on rows i, i+1 with partial pivoting
  double c0 = dd[0], c1 = du[0], c2 = 0.0;   // current row i: (c0 at col i, c1 at i+1, c2 at i+2)
  for (int i = 0; i < k - 1; ++i) {
    double r0 = dl[i], r1 = dd[i + 1], r2 = i + 1 < k - 1 ? du[i + 1] : 0.0;   // row i+1 at cols i, i+1, i+2
    if (fabs(r0) > fabs(c0)) {   // swap rows
      piv[i] = 1;
      std::swap(c0, r0);
      std::swap(c1, r1);
      std::swap(c2, r2);
    }
    if (c0 == 0.0) c0 = 1e-300;
    m[i] = r0 / c0;
    u0[i] = c0;
    u1[i] = c1;
    u2[i] = c2;
    c0 = r1 - m[i] * c1;
    c1 = r2 - m[i] * c2;
    c2 = 0.0;
  }
  u0[k - 1] = c0 == 0.0 ? 1e-300 : c0;
  u1[k - 1] = 0.0;
  u2[k - 1] = 0.0;
  for (int rep = 0; rep < 3; ++rep) {
    // forward: apply L^-1 with the recorded swaps
    for (int i = 0; i < k - 1; ++i) {
      if (piv[i]) std::swap(v[i], v[i + 1]);
      v[i + 1] -= m[i] * v[i];
    }
    // backward: U x = v
    for (int i = k - 1; i >= 0; --i) {
      double s = v[i];
      if (i + 1 < k) s -= u1[i] * v[i + 1];
      if (i + 2 < k) s -= u2[i] * v[i + 2];
      v[i] = s / u0[i];
    }
    double nrm = 0.0;
    for (double x : v) nrm += x * x;
    nrm = sqrt(nrm);
    for (double &x : v) x /= nrm;
  }
  for (int i = 0; i < k; ++i)
    if (v[i] != 0.0) {
      if (v[i] < 0) for (double &x : v) x = -x;
      break;
    }
  return v;
}

// All eigenvalues of T in ascending order: the i-th is the smallest x with at least i + 1
// eigenvalues below it, found by bisection on the Sturm count inside the Gershgorin interval.
std::vector<double> tridiag_all(const double *a, const double *b, int k) {
  std::vector<double> ev(k);
  if (k <= 0) return ev;
  double glo = INFINITY, ghi = -INFINITY;
  for (int i = 0; i < k; ++i) {
    const double r = (i ? fabs(b[i - 1]) : 0.0) + (i < k - 1 ? fabs(b[i]) : 0.0);
    glo = fmin(glo, a[i] - r);
    ghi = fmax(ghi, a[i] + r);
  }
  for (int j = 0; j < k; ++j) {
    double lo = j ? ev[j - 1] : glo, hi = ghi;   // eigenvalues are sorted: start at the previous one
    if (sturm_count(a, b, k, lo) >= j + 1) lo = glo;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (sturm_count(a, b, k, mid) >= j + 1) hi = mid; else lo = mid;
    }
    ev[j] = 0.5 * (lo + hi);
  }
  return ev;
}

double psi_eigenvalue(hub_ctx *h, double E0) {
  double v = E0;
  const int k = (int)h->alpha.size();
  if (h->psi_at_target && k > 0) {
    const std::vector<double> ev = tridiag_all(h->alpha.data(), h->beta.data(), k);
    v = ev[0];
    for (double e : ev)
      if (fabs(e - h->psi_target) < fabs(v - h->psi_target)) v = e;
  }
  h->psi_value = v;
  return v;
}

// In the k = 0 sector the start vector is projected onto the sector (ties of the short rows)
// in w, which then stands for it.
static int k0_start(hub_ctx *h, const double **x0, double *w, cudaStream_t s) {
  if (!h->k0) return HUB_OK;
  if (*x0 != w) HUB_CUDA(cudaMemcpyAsync(w, *x0, sizeof(double) * vec_len(h), cudaMemcpyDeviceToDevice, s));
  *x0 = w;
  return k0_project_inplace(h, w, s);
}

static int ensure_workspace(hub_ctx *h, int64_t D) {
  for (int k = 0; k < 3; ++k)
    if (!h->work[k] && !dev_alloc((void **)&h->work[k], sizeof(double) * D, "Lanczos vector")) return HUB_ERR_OOM;
  if (!h->d_scal && !dev_alloc((void **)&h->d_scal, sizeof(double) * 8, "Lanczos scalars")) return HUB_ERR_OOM;
  if (!h->h_scal) HUB_CUDA(cudaMallocHost((void **)&h->h_scal, sizeof(double) * 8));
  return ensure_partials(h, vec_grid());
}

}  // namespace hub

using namespace hub;

extern "C" int hub_lanczos_ground(hub_t h, const double *x0_dev, int maxit, double tol, double *E0,
                                  double *psi_dev, int *iters, void *stream) {
  int rc = ready(h, "hub_lanczos_ground");
  if (rc) return rc;
  if (!E0) return fail(HUB_ERR_ARG, "hub_lanczos_ground: E0 is NULL");
  if (maxit < 1) return fail(HUB_ERR_ARG, "hub_lanczos_ground: maxit < 1");
  const int64_t D = vec_len(h);
  if (D == 0) return fail(HUB_ERR_ARG, "hub_lanczos_ground: empty sector");
  if (small_eligible(h)) return small_lanczos(h, x0_dev, maxit, tol, E0, psi_dev, iters, (cudaStream_t)stream);
  if (use_fast(h)) {
    if (!x0_dev) {
      // the fast driver converts an FP64 start vector: draw it into the FP64 workspace
      if (!h->work[2] && !dev_alloc((void **)&h->work[2], sizeof(double) * D, "start vector")) return HUB_ERR_OOM;
      k_splitmix_uniform<<<vec_grid(), kVecThreads, 0, (cudaStream_t)stream>>>(D, h->work[2]);
      HUB_LAUNCH_CHECK();
      x0_dev = h->work[2];
    }
    return fast_lanczos(h, x0_dev, maxit, tol, E0, psi_dev, iters, (cudaStream_t)stream);
  }
  rc = ensure_workspace(h, D);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int G = vec_grid(), T = kVecThreads;
  double *qp = h->work[0], *q = h->work[1], *w = h->work[2];
  double *scal = h->d_scal, *P = h->partials;

  // q_1 = x0 / |x0|
  const double *x0 = x0_dev;
  if (!x0) {
    k_splitmix_uniform<<<G, T, 0, s>>>(D, w);
    HUB_LAUNCH_CHECK();
    x0 = w;
  }
  if ((rc = k0_start(h, &x0, w, s))) return rc;
  count_launch(h, x0_dev ? 3 : 4);   // [splitmix], dot, reduce, copy_scaled
  k_dot<<<G, T, 0, s>>>(D, x0, x0, P);
  HUB_LAUNCH_CHECK();
  if ((rc = reduce_partials(P, G, scal + 3, 1, s))) return rc;
  k_copy_scaled<<<G, T, 0, s>>>(D, q, x0, scal + 3);
  HUB_CUDA(cudaMemsetAsync(qp, 0, sizeof(double) * D, s));
  HUB_CUDA(cudaMemsetAsync(scal + 2, 0, sizeof(double), s));
  HUB_CUDA(cudaMemcpyAsync(h->h_scal + 3, scal + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
  HUB_CUDA(cudaStreamSynchronize(s));
  h->start_norm = h->h_scal[3];
  if (!(h->h_scal[3] > 0.0) || !std::isfinite(h->h_scal[3]))
    return fail(HUB_ERR_ARG, "hub_lanczos_ground: start vector is zero or not finite");

  h->alpha.clear();
  h->beta.clear();
  double E = 0.0, E_prev = 0.0;
  LowestTracker lowest;
  int status = HUB_ERR_NOCONV;
  for (int j = 0; j < maxit; ++j) {
    if ((rc = apply_launch(h, q, w, s))) return rc;
    count_launch(h, 5);   // sub_dot, reduce, sub_norm, reduce, scale_inv
    k_sub_dot<<<G, T, 0, s>>>(D, w, qp, q, scal + 2, P);
    HUB_LAUNCH_CHECK();
    if ((rc = reduce_partials(P, G, scal + 0, 0, s))) return rc;
    k_sub_norm<<<G, T, 0, s>>>(D, w, q, scal + 0, P);
    HUB_LAUNCH_CHECK();
    if ((rc = reduce_partials(P, G, scal + 1, 1, s))) return rc;
    HUB_CUDA(cudaMemcpyAsync(h->h_scal, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    HUB_CUDA(cudaStreamSynchronize(s));
    const double a = h->h_scal[0], b = h->h_scal[1];
    if (!std::isfinite(a) || !std::isfinite(b)) return fail(HUB_ERR_CUDA, "hub_lanczos_ground: non-finite alpha/beta");
    h->alpha.push_back(a);
    h->beta.push_back(b);
    if (tol > 0) E = lowest.next(h->alpha.data(), h->beta.data(), (int)h->alpha.size());   // else at the end
    if (tol > 0 && j > 0 && fabs(E - E_prev) < tol) {
      status = HUB_OK;
      break;
    }
    E_prev = E;
    if (b <= 1e-14 * fmax(1.0, fabs(a))) {
      status = HUB_CONVERGED_BREAKDOWN;
      break;
    }
    if (j + 1 < maxit) {
      k_scale_inv<<<G, T, 0, s>>>(D, w, scal);
      HUB_LAUNCH_CHECK();
      double *t0 = qp;
      qp = q;
      q = w;
      w = t0;
    }
  }
  if (tol <= 0 && status == HUB_ERR_NOCONV) status = HUB_OK;
  if (tol <= 0) E = tridiag_lowest(h->alpha.data(), h->beta.data(), (int)h->alpha.size());
  *E0 = E;
  const int k = (int)h->alpha.size();
  if (iters) *iters = k;

  if (psi_dev) {
    // second pass: psi = sum_j v_j q_j with v the lowest eigenvector of T_k
    std::vector<double> v = tridiag_vector(h->alpha.data(), h->beta.data(), k, psi_eigenvalue(h, E));
    qp = h->work[0];
    q = h->work[1];
    w = h->work[2];
    const double *xs = x0_dev;
    if (!xs) {
      k_splitmix_uniform<<<G, T, 0, s>>>(D, w);
      HUB_LAUNCH_CHECK();
      xs = w;
    }
    if ((rc = k0_start(h, &xs, w, s))) return rc;
    k_copy_scaled<<<G, T, 0, s>>>(D, q, xs, scal + 3);
    HUB_CUDA(cudaMemsetAsync(qp, 0, sizeof(double) * D, s));
    HUB_CUDA(cudaMemsetAsync(psi_dev, 0, sizeof(double) * D, s));
    for (int j = 0; j < k; ++j) {
      k_axpy<<<G, T, 0, s>>>(D, v[j], q, psi_dev);
      HUB_LAUNCH_CHECK();
      if (j + 1 == k) break;
      if ((rc = apply_launch(h, q, w, s))) return rc;
      k_recur<<<G, T, 0, s>>>(D, w, q, qp, h->alpha[j], j ? h->beta[j - 1] : 0.0, 1.0 / h->beta[j]);
      HUB_LAUNCH_CHECK();
      double *t0 = qp;
      qp = q;
      q = w;
      w = t0;
    }
    // normalise psi
    k_dot<<<G, T, 0, s>>>(D, psi_dev, psi_dev, P);
    HUB_LAUNCH_CHECK();
    if ((rc = reduce_partials(P, G, scal + 4, 1, s))) return rc;
    k_scale_by<<<G, T, 0, s>>>(D, psi_dev, scal + 4);
    HUB_LAUNCH_CHECK();
    HUB_CUDA(cudaStreamSynchronize(s));
  }
  if (status == HUB_ERR_NOCONV) set_error("hub_lanczos_ground: maxit reached before |dE0| < tol");
  return status;
}

extern "C" int hub_lanczos_coeffs(hub_t h, double *alpha_host, double *beta_host, int cap, int *n) {
  if (!h) return fail(HUB_ERR_ARG, "hub_lanczos_coeffs: NULL handle");
  int k = (int)h->alpha.size();
  if (n) *n = k;
  for (int i = 0; i < k && i < cap; ++i) {
    if (alpha_host) alpha_host[i] = h->alpha[i];
    if (beta_host) beta_host[i] = i < (int)h->beta.size() ? h->beta[i] : 0.0;   // last beta may be unknown
  }
  return HUB_OK;
}

extern "C" int hub_lanczos_spectrum(hub_t h, const double *x0_dev, int maxit, int n_eig, double *eig_host,
                                    double *resid_host, int *n_found, void *stream) {
  if (!h) return fail(HUB_ERR_ARG, "hub_lanczos_spectrum: NULL handle");
  if (n_eig < 1 || !eig_host || !n_found || maxit < 1 || maxit > 3000)
    return fail(HUB_ERR_ARG, "hub_lanczos_spectrum: bad argument");
  double E0 = 0.0;
  int it = 0;
  int rc = hub_lanczos_ground(h, x0_dev, maxit, 0.0, &E0, nullptr, &it, stream);
  if (rc < 0) return rc;
  const int k = (int)h->alpha.size();
  const double *a = h->alpha.data();
  std::vector<double> b(h->beta.begin(), h->beta.end());
  b.resize(k, 0.0);
  const std::vector<double> mu = tridiag_all(a, b.data(), k);
  const std::vector<double> nu = k > 1 ? tridiag_all(a + 1, b.data() + 1, k - 1) : std::vector<double>();
  double scale = 1.0;
  for (double m : mu) scale = fmax(scale, fabs(m));
  const double tol = 1e-10 * scale;
  // Cullum-Willoughby: numerically multiple eigenvalues of T are kept once; a simple one is
  // spurious if the matrix without its first row and column has it as well.
  std::vector<double> good;
  for (int i = 0; i < k;) {
    int j = i + 1;
    while (j < k && mu[j] - mu[j - 1] <= tol) ++j;
    const double m = mu[i];
    bool keep = j - i > 1;
    if (!keep) {
      keep = true;
      const auto p = std::lower_bound(nu.begin(), nu.end(), m - tol);
      if (p != nu.end() && *p <= m + tol) keep = false;
    }
    if (keep) good.push_back(m);
    i = j;
  }
  const int n = std::min<int>(n_eig, (int)good.size());
  for (int i = 0; i < n; ++i) {
    eig_host[i] = good[i];
    if (resid_host) {
      // |H y - theta y| for the Ritz pair: beta_{k-1} times the last component of T's eigenvector
      const std::vector<double> v = tridiag_vector(a, b.data(), k, good[i]);
      resid_host[i] = fabs(b[k - 1] * v[k - 1]);
    }
  }
  *n_found = n;
  return HUB_OK;
}

extern "C" int hub_lanczos_ritz(hub_t h, const double *x0_dev, int maxit, double target, double *psi_dev,
                                double *ritz_host, void *stream) {
  if (!h) return fail(HUB_ERR_ARG, "hub_lanczos_ritz: NULL handle");
  if (!psi_dev || !ritz_host || maxit < 1 || maxit > 3000 || !std::isfinite(target))
    return fail(HUB_ERR_ARG, "hub_lanczos_ritz: bad argument");
  h->psi_at_target = true;
  h->psi_target = target;
  double E0 = 0.0;
  int it = 0;
  const int rc = hub_lanczos_ground(h, x0_dev, maxit, 0.0, &E0, psi_dev, &it, stream);
  h->psi_at_target = false;
  if (rc < 0) return rc;
  *ritz_host = h->psi_value;
  return HUB_OK;
}
