// hub_batch.cu -- many small ground-state problems in one persistent launch (K6).
//
// Sec. VIII: an exact-diagonalisation impurity solver repeats the ground-state search for
// every (N_up, N_dn) sector and every bath-parameter set.  Each such problem is small (for
// an 8-site impurity star the largest sector has 70 x 70 = 4900 states), so one problem per
// launch would be dominated by launch and synchronisation latency.  Here all problems are
// jobs of one kernel: persistent CTAs take jobs from an atomic queue (largest first), keep
// the job's three Lanczos vectors in shared memory and run the whole plain Lanczos
// iteration of Sec. IV / V inside the CTA.  The matrix-free product is Eq. 11 on the
// count_dn x count_up state matrix (Eq. count2): spin-up hops gather inside a row, spin-down
// hops combine rows, the diagonal comes from the set bits of I_up & I_dn (Sec. III.B); the
// hopping values -t_b * esign (Eq. 8) are formed on the fly from the job's parameter set.
// The one-spin bases and hopping structures for every N = 0..M are built once by the
// regular set-up kernels (hub_basis / hub_hopping) and shared by all jobs.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "hub_internal.cuh"

namespace hub {

constexpr int kBatchMaxSites = 16;
constexpr int kBatchMaxDim = 8192;      // three FP64 vectors of this length in shared memory
#ifndef HUB_BATCH_THREADS
#define HUB_BATCH_THREADS 512            // threads per CTA (one job per CTA at a time)
#endif
constexpr int kBatchThreads = HUB_BATCH_THREADS;
constexpr int kBatchCheckEvery = 8;     // E0 of T_j is evaluated every this many iterations
#ifndef HUB_BATCH_SPLIT
#define HUB_BATCH_SPLIT 2048              // jobs of at most this many states run in a second launch
#endif
constexpr int kBatchSplit = HUB_BATCH_SPLIT;

struct BatchTables {
  const uint32_t *basis;     // all one-spin bases, N = 0..M, concatenated
  const int32_t *rp;         // row pointers (global entry offsets), concatenated
  const uint32_t *scol;      // column | sign bit, entries concatenated
  const uint8_t *bond;       // bond id per entry
  int off_basis[kBatchMaxSites + 2];   // start of N's basis in `basis`
  int off_rp[kBatchMaxSites + 2];      // start of N's row pointers in `rp`
  int count[kBatchMaxSites + 1];       // C(M, N)
};

struct BatchArgs {
  int M, n_bonds, n_jobs, maxit;
  double tol;
  const double *t, *U, *eps;           // per parameter set: [n_bonds], [M], [M] (eps may be null)
  const int32_t *job_nup, *job_ndn, *job_param, *order;
  int *counter;                        // work queue head (zeroed before the launch)
  double *E0;
  int32_t *iters, *status;
};

__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();                     // red may still be read from the previous call
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k < nw; ++k) s += red[k];   // every thread, same fixed order
  return s;
}

// Number of eigenvalues of the tridiagonal (a, b) smaller than x (Sturm sequence).
__device__ int sturm_count_dev(const double *a, const double *b, int k, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < k; ++i) {
    const double bb = i ? b[i - 1] * b[i - 1] : 0.0;
    d = (a[i] - x) - (i ? bb / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

// Lowest eigenvalue of the k x k tridiagonal by 32-way multisection, one warp.
__device__ double tri_lowest_warp(const double *a, const double *b, int k) {
  const int lane = threadIdx.x & 31;
  double lo = INFINITY, hi = -INFINITY;
  for (int i = lane; i < k; i += 32) {
    const double r = (i ? fabs(b[i - 1]) : 0.0) + (i < k - 1 ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if (k == 1) return a[0];
  for (int round = 0; round < 16; ++round) {
    const double step = (hi - lo) / 32.0;
    const double x = lane == 31 ? hi : lo + step * (lane + 1);
    const unsigned ball = __ballot_sync(0xffffffffu, sturm_count_dev(a, b, k, x) >= 1);
    const int L = ball ? __ffs(ball) - 1 : 31;
    const double nhi = __shfl_sync(0xffffffffu, x, L);
    const double nlo = L == 0 ? lo : __shfl_sync(0xffffffffu, x, L - 1);
    if (!(nhi < hi || nlo > lo)) break;        // no progress at double precision
    lo = nlo;
    hi = nhi;
  }
  return 0.5 * (lo + hi);
}

__global__ void __launch_bounds__(kBatchThreads) k_batch_lanczos(const BatchTables T, const BatchArgs A) {
  extern __shared__ __align__(16) double sm[];
  __shared__ double red[32];
  __shared__ double s_par[3][kBatchMaxSites > 64 ? kBatchMaxSites : 64];
  __shared__ double s_t[kMaxBonds];
  __shared__ int s_job, s_stop;
  __shared__ double s_E;
  // layout: q_prev | q | w (Dmax each), alpha | beta (maxit each)
  const int Dmax = kBatchMaxDim;
  (void)Dmax;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) s_job = atomicAdd(A.counter, 1);
    __syncthreads();
    const int slot = s_job;
    if (slot >= A.n_jobs) return;
    const int job = A.order[slot];
    const int Nu = A.job_nup[job], Nd = A.job_ndn[job], P = A.job_param[job];
    const int nu = T.count[Nu], nd = T.count[Nd], D = nu * nd;
    double *qp = sm, *q = sm + D, *w = sm + 2 * D;
    double *alpha = sm + 3 * D, *beta = alpha + A.maxit;
    for (int i = tid; i < A.n_bonds; i += blockDim.x) s_t[i] = A.t[(int64_t)P * A.n_bonds + i];
    for (int i = tid; i < A.M; i += blockDim.x) {
      s_par[0][i] = A.U[(int64_t)P * A.M + i];
      s_par[1][i] = A.eps ? A.eps[(int64_t)P * A.M + i] : 0.0;
    }
    const uint32_t *bu = T.basis + T.off_basis[Nu], *bd = T.basis + T.off_basis[Nd];
    const int32_t *rpu = T.rp + T.off_rp[Nu], *rpd = T.rp + T.off_rp[Nd];
    // start vector: SplitMix64 uniform [-1, 1) with counter (job << 32) | (element + 1)
    double nrm = 0.0;
    for (int n = tid; n < D; n += blockDim.x) {
      uint64_t z = (((uint64_t)job << 32) | (uint64_t)(n + 1)) * 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      const double v = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
      q[n] = v;
      qp[n] = 0.0;
      nrm = fma(v, v, nrm);
    }
    __syncthreads();
    nrm = sqrt(block_sum(nrm, red));
    const double inv0 = 1.0 / nrm;
    for (int n = tid; n < D; n += blockDim.x) q[n] *= inv0;
    double b_prev = 0.0, E_prev = 0.0, E = 0.0;
    int status = HUB_ERR_NOCONV, j = 0;
    if (tid == 0) s_stop = 0;
    for (j = 0; j < A.maxit; ++j) {
      __syncthreads();
      // w = H q - beta_{j-1} q_{j-1}; alpha = <q, w>
      double dot = 0.0;
      for (int n = tid; n < D; n += blockDim.x) {
        const int d = n / nu, u = n - d * nu;
        const uint32_t Iu = bu[u], Id = bd[d];
        double dg = 0.0;
        for (uint32_t m = Iu & Id; m; m &= m - 1) dg += s_par[0][__ffs(m) - 1];
        for (uint32_t m = Iu; m; m &= m - 1) dg += s_par[1][__ffs(m) - 1];
        for (uint32_t m = Id; m; m &= m - 1) dg += s_par[1][__ffs(m) - 1];
        double acc = dg * q[n];
        for (int k = rpu[u]; k < rpu[u + 1]; ++k) {
          const uint32_t sc = T.scol[k];
          const double v = q[d * nu + (int)(sc & 0x7fffffffu)];
          acc = fma((sc >> 31) ? s_t[T.bond[k]] : -s_t[T.bond[k]], v, acc);
        }
        for (int k = rpd[d]; k < rpd[d + 1]; ++k) {
          const uint32_t sc = T.scol[k];
          const double v = q[(int)(sc & 0x7fffffffu) * nu + u];
          acc = fma((sc >> 31) ? s_t[T.bond[k]] : -s_t[T.bond[k]], v, acc);
        }
        acc = fma(-b_prev, qp[n], acc);
        w[n] = acc;
        dot = fma(q[n], acc, dot);
      }
      const double a = block_sum(dot, red);
      double nn = 0.0;
      for (int n = tid; n < D; n += blockDim.x) {
        const double v = fma(-a, q[n], w[n]);
        w[n] = v;
        nn = fma(v, v, nn);
      }
      const double b = sqrt(block_sum(nn, red));
      if (tid == 0) {
        alpha[j] = a;
        beta[j] = b;
      }
      const bool breakdown = b <= 1e-14 * fmax(1.0, fabs(a));
      const bool check = breakdown || j + 1 == A.maxit || ((j + 1) % kBatchCheckEvery == 0);
      __syncthreads();
      if (check) {
        if (tid < 32) {
          const double e = tri_lowest_warp(alpha, beta, j + 1);
          if (tid == 0) {
            s_E = e;
            int stop = 0;
            if (breakdown) stop = 2;
            else if (A.tol > 0 && j + 1 > kBatchCheckEvery && fabs(e - E_prev) < A.tol) stop = 1;
            s_stop = stop;
          }
        }
        __syncthreads();
        E = s_E;
        if (s_stop) {
          status = s_stop == 2 ? HUB_CONVERGED_BREAKDOWN : HUB_OK;
          ++j;
          break;
        }
        E_prev = E;
      }
      // q_{j+1} = w / beta; rotate (q_prev <- q, q <- w, w <- old q_prev)
      const double ib = 1.0 / b;
      for (int n = tid; n < D; n += blockDim.x) w[n] *= ib;
      double *t0 = qp;
      qp = q;
      q = w;
      w = t0;
      b_prev = b;
    }
    if (A.tol <= 0 && status == HUB_ERR_NOCONV) status = HUB_OK;
    if (tid == 0) {
      A.E0[job] = E;
      A.iters[job] = j > A.maxit ? A.maxit : j;
      A.status[job] = status;
    }
    __syncthreads();
  }
}

}  // namespace hub

using namespace hub;

extern "C" int hub_batch_ground(int M, int n_bonds, const int32_t *bonds_host, int n_params, const double *t_host,
                                const double *U_host, const double *eps_host, int n_jobs, const int32_t *job_nup,
                                const int32_t *job_ndn, const int32_t *job_param, int maxit, double tol,
                                double *E0_host, int32_t *iters_host, int32_t *status_host, void *stream) {
  if (M < 1 || M > kBatchMaxSites) return fail(HUB_ERR_ARG, "hub_batch_ground: need 1 <= M <= 16");
  if (n_params < 1 || n_jobs < 0 || maxit < 1 || maxit > 1000)
    return fail(HUB_ERR_ARG, "hub_batch_ground: need n_params >= 1, n_jobs >= 0, 1 <= maxit <= 1000");
  if (!t_host || !U_host || (n_jobs && (!job_nup || !job_ndn || !job_param || !E0_host || !iters_host || !status_host)))
    return fail(HUB_ERR_ARG, "hub_batch_ground: NULL argument");
  if (n_jobs == 0) return HUB_OK;
  std::vector<int> cnt(M + 1);
  for (int N = 0; N <= M; ++N) {
    double c = 1.0;
    for (int k = 1; k <= N; ++k) c = c * (M - N + k) / k;
    cnt[N] = (int)std::llround(c);
  }
  int Dmax = 1;
  for (int k = 0; k < n_jobs; ++k) {
    const int a = job_nup[k], b = job_ndn[k], p = job_param[k];
    if (a < 0 || a > M || b < 0 || b > M || p < 0 || p >= n_params)
      return fail(HUB_ERR_ARG, "hub_batch_ground: job " + std::to_string(k) + " has a bad sector or parameter set");
    const int64_t D = (int64_t)cnt[a] * cnt[b];
    if (D > kBatchMaxDim)
      return fail(HUB_ERR_ARG, "hub_batch_ground: job " + std::to_string(k) + " has dimension " + std::to_string(D) +
                                   " > 8192; use hub_lanczos_ground");
    Dmax = std::max<int>(Dmax, (int)D);
  }
  for (int k = 0; k < n_params * M; ++k)
    if (!(U_host[k] == U_host[k])) return fail(HUB_ERR_ARG, "hub_batch_ground: U is NaN");

  // one-spin bases and hopping structures for every N, built by the regular set-up kernels
  std::vector<double> ones(std::max(n_bonds, 1), 1.0);
  std::vector<uint32_t> basis;
  std::vector<int32_t> rp;
  std::vector<uint32_t> scol;
  std::vector<uint8_t> bond;
  BatchTables T{};
  for (int N = 0; N <= M; ++N) {
    hub_t h = nullptr;
    int rc = hub_basis(M, N, N, &h);
    if (rc) return rc;
    rc = hub_hopping(h, n_bonds, bonds_host, ones.data(), nullptr);
    if (rc) {
      hub_free(h);
      return rc;
    }
    const int64_t n = h->count[0];
    const SpinCSR &c = h->csr[0];
    std::vector<uint32_t> b(n);
    std::vector<int32_t> r(n + 1);
    std::vector<uint32_t> sc(c.nnz);
    std::vector<uint8_t> bo(c.nnz);
    cudaError_t e = cudaMemcpy(b.data(), h->basis[0], sizeof(uint32_t) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(r.data(), c.rowptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && c.nnz) e = cudaMemcpy(sc.data(), c.scol, sizeof(uint32_t) * c.nnz, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && c.nnz) e = cudaMemcpy(bo.data(), c.bond, c.nnz, cudaMemcpyDeviceToHost);
    hub_free(h);
    if (e != cudaSuccess) return cuda_fail(e, "batched set-up copy", __FILE__, __LINE__);
    T.off_basis[N] = (int)basis.size();
    T.off_rp[N] = (int)rp.size();
    T.count[N] = (int)n;
    const int base = (int)scol.size();
    basis.insert(basis.end(), b.begin(), b.end());
    for (int32_t v : r) rp.push_back(v + base);
    scol.insert(scol.end(), sc.begin(), sc.end());
    bond.insert(bond.end(), bo.begin(), bo.end());
  }
  // largest jobs first
  std::vector<int32_t> order(n_jobs);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return (int64_t)cnt[job_nup[a]] * cnt[job_ndn[a]] > (int64_t)cnt[job_nup[b]] * cnt[job_ndn[b]];
  });

  // device copies of everything (freed before returning)
  std::vector<void *> owned;
  auto up = [&](const void *src, size_t bytes, const char *what) -> void * {
    void *p = nullptr;
    if (!dev_alloc(&p, bytes, what)) return nullptr;
    owned.push_back(p);
    if (src && cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
    return p;
  };
  auto release = [&]() {
    for (void *p : owned) dev_free(p);
  };
  BatchArgs A{};
  A.M = M;
  A.n_bonds = n_bonds;
  A.n_jobs = n_jobs;
  A.maxit = maxit;
  A.tol = tol;
  T.basis = (const uint32_t *)up(basis.data(), sizeof(uint32_t) * basis.size(), "batch bases");
  T.rp = (const int32_t *)up(rp.data(), sizeof(int32_t) * rp.size(), "batch row pointers");
  T.scol = (const uint32_t *)up(scol.data(), sizeof(uint32_t) * std::max<size_t>(scol.size(), 1), "batch columns");
  T.bond = (const uint8_t *)up(bond.data(), std::max<size_t>(bond.size(), 1), "batch bond ids");
  A.t = (const double *)up(t_host, sizeof(double) * std::max(n_params * n_bonds, 1), "batch t");
  A.U = (const double *)up(U_host, sizeof(double) * n_params * M, "batch U");
  A.eps = eps_host ? (const double *)up(eps_host, sizeof(double) * n_params * M, "batch eps") : nullptr;
  A.job_nup = (const int32_t *)up(job_nup, sizeof(int32_t) * n_jobs, "batch jobs");
  A.job_ndn = (const int32_t *)up(job_ndn, sizeof(int32_t) * n_jobs, "batch jobs");
  A.job_param = (const int32_t *)up(job_param, sizeof(int32_t) * n_jobs, "batch jobs");
  A.order = (const int32_t *)up(order.data(), sizeof(int32_t) * n_jobs, "batch order");
  A.counter = (int *)up(nullptr, 2 * sizeof(int), "batch queues");
  A.E0 = (double *)up(nullptr, sizeof(double) * n_jobs, "batch E0");
  A.iters = (int32_t *)up(nullptr, sizeof(int32_t) * n_jobs, "batch iterations");
  A.status = (int32_t *)up(nullptr, sizeof(int32_t) * n_jobs, "batch status");
  if (!T.basis || !T.rp || !T.scol || !T.bond || !A.t || !A.U || (eps_host && !A.eps) || !A.job_nup || !A.job_ndn ||
      !A.job_param || !A.order || !A.counter || !A.E0 || !A.iters || !A.status) {
    release();
    return fail(HUB_ERR_OOM, "hub_batch_ground: device allocation or upload failed");
  }
  // The shared memory of a CTA holds three vectors of the largest job it may take, so one
  // launch for every job would give the small ones the large ones' footprint (one CTA per SM
  // at the impurity star's 4900 states).  Jobs of at most kBatchSplit states (a suffix of
  // the largest-first order) therefore run in a second launch on a second stream, sized for
  // them, whose CTAs fill the SMs beside the large jobs' (two independent queues, no waits
  // between the launches).
  cudaStream_t s = (cudaStream_t)stream;
  auto dim_of = [&](int32_t j) { return (int64_t)cnt[job_nup[j]] * cnt[job_ndn[j]]; };
  int n_large = 0;
  while (n_large < n_jobs && dim_of(order[n_large]) > kBatchSplit) ++n_large;
  if (n_large == 0 || n_large == n_jobs) n_large = n_jobs;        // one size class: one launch
  struct Part {
    int first, count, dmax;
  } parts[2] = {{0, n_large, Dmax}, {n_large, n_jobs - n_large, n_large < n_jobs ? (int)dim_of(order[n_large]) : 0}};
  const int n_parts = n_large < n_jobs ? 2 : 1;
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev_ready = nullptr, ev_done = nullptr;
  int rc = HUB_OK;
  cudaError_t e = cudaMemsetAsync(A.counter, 0, 2 * sizeof(int), s);
  if (e == cudaSuccess && n_parts == 2) {
    e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev_ready, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, ev_ready, 0);
  }
  size_t smem_max = 0;
  for (int p = 0; p < n_parts; ++p)
    smem_max = std::max(smem_max, sizeof(double) * (3 * (size_t)parts[p].dmax + 2 * (size_t)maxit));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_batch_lanczos, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
  for (int p = 0; p < n_parts && e == cudaSuccess; ++p) {
    const size_t smem = sizeof(double) * (3 * (size_t)parts[p].dmax + 2 * (size_t)maxit);
    int per_sm = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_lanczos, kBatchThreads, smem);
    if (e != cudaSuccess) break;
    BatchArgs Ap = A;
    Ap.n_jobs = parts[p].count;
    Ap.order = A.order + parts[p].first;
    Ap.counter = A.counter + p;
    const int grid = std::max(1, std::min(parts[p].count, num_sms() * std::max(per_sm, 1)));
    k_batch_lanczos<<<grid, kBatchThreads, smem, p == 0 ? s : s2>>>(T, Ap);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && n_parts == 2) e = cudaEventRecord(ev_done, s2);
  if (e == cudaSuccess && n_parts == 2) e = cudaStreamWaitEvent(s, ev_done, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(E0_host, A.E0, sizeof(double) * n_jobs, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(iters_host, A.iters, sizeof(int32_t) * n_jobs, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(status_host, A.status, sizeof(int32_t) * n_jobs, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) rc = cuda_fail(e, "hub_batch_ground", __FILE__, __LINE__);
  if (s2) {
    cudaStreamSynchronize(s2);         // nothing of this call may outlive it
    cudaStreamDestroy(s2);
  }
  if (ev_ready) cudaEventDestroy(ev_ready);
  if (ev_done) cudaEventDestroy(ev_done);
  release();
  if (rc) return rc;
  for (int k = 0; k < n_jobs; ++k)
    if (status_host[k] == HUB_ERR_NOCONV) {
      set_error("hub_batch_ground: some jobs reached maxit before |dE0| < tol");
      return HUB_ERR_NOCONV;
    }
  return HUB_OK;
}
