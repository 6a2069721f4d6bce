// hub_setup.cu -- sector set-up: one-spin bases by combinadic unranking (K1) and the
// one-spin hopping matrices in CSR form (K2), plus the handle's accessors.
//
// Sec. II (Eqs. count2, count3, Appendix A): the spin-sigma basis is the ascending list of
// M-bit strings with N_sigma bits set.  Algorithm I finds it by scanning every integer
// between the smallest and the largest such string; here thread r computes the r-th
// string directly from the combinatorial number system, which yields the same order.
// Sec. III.A (Eq. 8) and Sec. IV.A (Eqs. 9-10): the hopping matrix of one spin holds,
// for each string s and each bond with exactly one end occupied, the element
// -t_b * esign with esign = (-1)^(electrons strictly between the two sites), at the
// column of the hopped string; that column is found by ranking instead of by a stored
// 2^M index table or a binary search.
#include <algorithm>
#include <cmath>
#include <new>
#include <cstdio>
#include <cstring>
#include <string>

#include "hub_internal.cuh"

namespace hub {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }
int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
  char buf[512];
  snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  g_err = buf;
  return e == cudaErrorMemoryAllocation ? HUB_ERR_OOM : HUB_ERR_CUDA;
}

bool dev_alloc(void **p, size_t bytes, const char *what) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char buf[256];
    snprintf(buf, sizeof buf, "cudaMalloc of %zu bytes for %s failed: %s", bytes, what,
             cudaGetErrorString(e));
    g_err = buf;
    *p = nullptr;
    return false;
  }
  return true;
}

void dev_free(void *p) {
  if (p) cudaFree(p);
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

int ensure_partials(hub_ctx *h, int64_t n) {
  if (h->partials_n >= n) return HUB_OK;
  dev_free(h->partials);
  h->partials = nullptr;
  h->partials_n = 0;
  if (!dev_alloc((void **)&h->partials, sizeof(double) * n, "reduction partials")) return HUB_ERR_OOM;
  h->partials_n = n;
  return HUB_OK;
}


// K1: thread r writes the r-th M-bit string with N ones in ascending order.  Walking from
// the top bit down, C(b, k) strings keep bit b clear with k ones left in bits 0..b-1, and
// all of them are smaller than any string with bit b set.
__global__ void k_unrank(int M, int N, int64_t count, const uint64_t *__restrict__ C,
                         uint32_t *__restrict__ out) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < count;
       r += (int64_t)gridDim.x * blockDim.x) {
    uint64_t rr = (uint64_t)r;
    uint32_t s = 0;
    int k = N;
    for (int b = M - 1; b >= 0 && k > 0; --b) {
      uint64_t c = C[b * kB + k];
      if (rr >= c) {
        s |= 1u << b;
        rr -= c;
        --k;
      }
    }
    out[r] = s;
  }
}

struct BondTable {
  int n;
  uint8_t i[kMaxBonds], j[kMaxBonds];
  double t[kMaxBonds];
};

__device__ __forceinline__ bool hop_of(uint32_t s, int i, int j, uint32_t *s2, int *sign) {
  if ((((s >> i) ^ (s >> j)) & 1u) == 0) return false;
  int lo = i < j ? i : j, hi = i < j ? j : i;
  uint32_t between = s & (((1u << hi) - 1u) ^ ((1u << (lo + 1)) - 1u));
  *sign = (__popc(between) & 1) ? -1 : 1;
  *s2 = s ^ (1u << i) ^ (1u << j);
  return true;
}

// K2a: number of allowed hops of each string.
__global__ void k_hop_count(int64_t count, const uint32_t *__restrict__ basis, BondTable bt,
                            int32_t *__restrict__ cnt) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < count;
       r += (int64_t)gridDim.x * blockDim.x) {
    uint32_t s = basis[r];
    int c = 0;
    for (int b = 0; b < bt.n; ++b) c += ((s >> bt.i[b]) ^ (s >> bt.j[b])) & 1u;
    cnt[r] = c;
  }
}

// Exclusive scan of cnt[0..n) into rowptr[0..n], one block; also the longest row.
__global__ void k_scan_rows(int64_t n, const int32_t *__restrict__ cnt, int32_t *__restrict__ rowptr,
                            int32_t *__restrict__ max_row) {
  __shared__ int64_t sums[1024];
  __shared__ int32_t mx[1024];
  const int T = blockDim.x, tid = threadIdx.x;
  int64_t chunk = (n + T - 1) / T;
  int64_t a = tid * chunk, b = min(n, a + chunk);
  int64_t s = 0;
  int32_t m = 0;
  for (int64_t r = a; r < b; ++r) {
    s += cnt[r];
    m = max(m, cnt[r]);
  }
  sums[tid] = s;
  mx[tid] = m;
  __syncthreads();
  if (tid == 0) {
    int64_t run = 0;
    int32_t mm = 0;
    for (int k = 0; k < T; ++k) {
      int64_t v = sums[k];
      sums[k] = run;
      run += v;
      mm = max(mm, mx[k]);
    }
    rowptr[n] = (int32_t)run;
    *max_row = mm;
  }
  __syncthreads();
  int64_t run = sums[tid];
  for (int64_t r = a; r < b; ++r) {
    rowptr[r] = (int32_t)run;
    run += cnt[r];
  }
}

// K2b: fill each row with its hops, columns ascending.
__global__ void k_hop_fill(int64_t count, const uint32_t *__restrict__ basis, BondTable bt,
                           const uint64_t *__restrict__ C, const int32_t *__restrict__ rowptr,
                           int32_t *__restrict__ col, double *__restrict__ val,
                           uint32_t *__restrict__ scol, uint8_t *__restrict__ bond) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < count;
       r += (int64_t)gridDim.x * blockDim.x) {
    uint32_t s = basis[r];
    int32_t base = rowptr[r];
    int k = 0;
    for (int b = 0; b < bt.n; ++b) {
      uint32_t s2;
      int sign;
      if (!hop_of(s, bt.i[b], bt.j[b], &s2, &sign)) continue;
      int32_t c = (int32_t)rank_of(s2, C);
      // insertion into the row, keeping columns ascending
      int p = k;
      while (p > 0 && col[base + p - 1] > c) {
        col[base + p] = col[base + p - 1];
        val[base + p] = val[base + p - 1];
        scol[base + p] = scol[base + p - 1];
        bond[base + p] = bond[base + p - 1];
        --p;
      }
      col[base + p] = c;
      val[base + p] = -bt.t[b] * (double)sign;
      scol[base + p] = (uint32_t)c | (sign < 0 ? 0x80000000u : 0u);
      bond[base + p] = (uint8_t)b;
      ++k;
    }
  }
}

// Per-string site-energy sum: sum_i eps_i * bit_i(s).
__global__ void k_eps_state(int64_t count, const uint32_t *__restrict__ basis, int M, const double *eps,
                            double *__restrict__ out) {
  __shared__ double e[kMaxSites];
  if (threadIdx.x < M) e[threadIdx.x] = eps[threadIdx.x];
  __syncthreads();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < count;
       r += (int64_t)gridDim.x * blockDim.x) {
    uint32_t s = basis[r];
    double v = 0.0;
    for (int i = 0; i < M; ++i)
      if ((s >> i) & 1u) v += e[i];
    out[r] = v;
  }
}

// Deterministic reduction of partials (fixed order): mode 0 -> sum, mode 1 -> sqrt(sum).
__global__ void k_reduce(const double *__restrict__ p, int n, double *__restrict__ out, int mode) {
  __shared__ double s[kReduceThreads];
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) v += p[k];
  s[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = mode == 1 ? sqrt(s[0]) : s[0];
}

// First stage for long partial lists: block b sums the contiguous chunk b (fixed order).
__global__ void k_reduce_chunks(const double *__restrict__ p, int n, int chunk, double *__restrict__ out) {
  __shared__ double s[kReduceThreads];
  const int a = blockIdx.x * chunk, b = min(n, a + chunk);
  double v = 0.0;
  for (int k = a + threadIdx.x; k < b; k += blockDim.x) v += p[k];
  s[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = s[0];
}

int reduce_partials(const double *partials, int n, double *out, int mode, cudaStream_t s) {
  k_reduce<<<1, kReduceThreads, 0, s>>>(partials, n, out, mode);
  HUB_LAUNCH_CHECK();
  return HUB_OK;
}

int reduce_partials_2stage(const double *partials, int n, double *tmp, int ntmp, double *out, int mode,
                           cudaStream_t s) {
  if (n <= 4 * kReduceThreads || ntmp < 2) return reduce_partials(partials, n, out, mode, s);
  const int chunks = std::min(ntmp, (n + 1023) / 1024);
  const int chunk = (n + chunks - 1) / chunks;
  const int nb = (n + chunk - 1) / chunk;
  k_reduce_chunks<<<nb, kReduceThreads, 0, s>>>(partials, n, chunk, tmp);
  HUB_LAUNCH_CHECK();
  k_reduce<<<1, kReduceThreads, 0, s>>>(tmp, nb, out, mode);
  HUB_LAUNCH_CHECK();
  return HUB_OK;
}

static int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  int64_t cap = (int64_t)num_sms() * 32;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

static void free_csr(SpinCSR &c) {
  dev_free(c.rowptr);
  dev_free(c.col);
  dev_free(c.val);
  dev_free(c.scol);
  dev_free(c.bond);
  c = SpinCSR{};
}

static int build_csr(hub_ctx *h, int spin, const BondTable &bt) {
  SpinCSR &c = h->csr[spin];
  free_csr(c);
  const int64_t n = h->count[spin];
  const int N = h->N[spin], M = h->M;
  // nnz = 2 * B * C(M-2, N-1) for 1 <= N <= M-1 (Sec. IV.A), zero otherwise
  int64_t nnz_expect = 0;
  if (N >= 1 && N <= M - 1 && M >= 2) {
    uint64_t c2 = 1;
    for (int k = 1; k <= N - 1; ++k) c2 = c2 * (uint64_t)(M - 2 - (N - 1) + k) / (uint64_t)k;
    nnz_expect = 2 * (int64_t)bt.n * (int64_t)c2;
  }
  if (nnz_expect > INT32_MAX) return fail(HUB_ERR_ARG, "hopping matrix has more than 2^31 nonzeros");
  int32_t *cnt = nullptr, *d_max = nullptr;
  if (!dev_alloc((void **)&c.rowptr, sizeof(int32_t) * (n + 1), "CSR rowptr") ||
      !dev_alloc((void **)&cnt, sizeof(int32_t) * n, "CSR counts") ||
      !dev_alloc((void **)&d_max, sizeof(int32_t), "CSR max row") ||
      !dev_alloc((void **)&c.col, sizeof(int32_t) * nnz_expect, "CSR cols") ||
      !dev_alloc((void **)&c.val, sizeof(double) * nnz_expect, "CSR vals") ||
      !dev_alloc((void **)&c.scol, sizeof(uint32_t) * nnz_expect, "CSR signed cols") ||
      !dev_alloc((void **)&c.bond, sizeof(uint8_t) * nnz_expect, "CSR bond ids")) {
    dev_free(cnt);
    dev_free(d_max);
    free_csr(c);
    return HUB_ERR_OOM;
  }
  int rc = HUB_OK;
  k_hop_count<<<grid_for(n, 256), 256>>>(n, h->basis[spin], bt, cnt);
  k_scan_rows<<<1, 1024>>>(n, cnt, c.rowptr, d_max);
  k_hop_fill<<<grid_for(n, 128), 128>>>(n, h->basis[spin], bt, h->binom, c.rowptr, c.col, c.val,
                                        c.scol, c.bond);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int32_t total = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&total, c.rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&c.max_row, d_max, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) rc = cuda_fail(e, "hopping CSR build", __FILE__, __LINE__);
  if (rc == HUB_OK && total != nnz_expect)
    rc = fail(HUB_ERR_CUDA, "hopping CSR nonzero count disagrees with 2*B*C(M-2,N-1)");
  c.nnz = total;
  dev_free(cnt);
  dev_free(d_max);
  if (rc != HUB_OK) free_csr(c);
  return rc;
}

}  // namespace hub

using namespace hub;

hub::Ham hub_ctx::view() const {
  Ham v{};
  v.M = M;
  v.n_up = count[0];
  v.n_dn = count[1];
  v.basis_up = basis[0];
  v.basis_dn = basis[1];
  const SpinCSR &cu = csr[0], &cd = csr[shared ? 0 : 1];
  v.rp_up = cu.rowptr;
  v.rp_dn = cd.rowptr;
  v.col_up = cu.col;
  v.col_dn = cd.col;
  v.val_up = cu.val;
  v.val_dn = cd.val;
  v.scol_up = cu.scol;
  v.scol_dn = cd.scol;
  v.eps_up = eps_state[0];
  v.eps_dn = eps_state[shared ? 0 : 1];
  v.has_eps = has_eps ? 1 : 0;
  v.uniform_U = uniform_U ? 1 : 0;
  v.U0 = U0;
  for (int i = 0; i < kMaxSites; ++i) v.U[i] = i < (int)U.size() ? U[i] : 0.0;
  v.uniform_t = 1;
  v.t0 = t.empty() ? 0.0 : t[0];
  for (double tb : t)
    if (tb != v.t0) v.uniform_t = 0;
  return v;
}

extern "C" const char *hub_last_error(void) { return g_err.c_str(); }

extern "C" int hub_basis(int M, int n_up, int n_dn, hub_t *out) {
  if (!out) return fail(HUB_ERR_ARG, "hub_basis: out is NULL");
  *out = nullptr;
  if (M < 1 || M > kMaxSites) return fail(HUB_ERR_ARG, "hub_basis: need 1 <= M <= 30");
  if (n_up < 0 || n_up > M || n_dn < 0 || n_dn > M)
    return fail(HUB_ERR_ARG, "hub_basis: need 0 <= n_up, n_dn <= M");
  hub_ctx *h = new (std::nothrow) hub_ctx();
  if (!h) return fail(HUB_ERR_OOM, "hub_basis: host allocation failed");
  HUB_CUDA(cudaGetDevice(&h->device));
  h->M = M;
  h->N[0] = n_up;
  h->N[1] = n_dn;
  h->shared = (n_up == n_dn);
  // Pascal triangle on the host (exact in uint64 for n <= 30)
  std::vector<uint64_t> C((size_t)kB * kB, 0);
  for (int n = 0; n < kB; ++n) {
    C[n * kB] = 1;
    for (int k = 1; k <= n; ++k) C[n * kB + k] = C[(n - 1) * kB + k - 1] + (k <= n - 1 ? C[(n - 1) * kB + k] : 0);
  }
  h->count[0] = (int64_t)C[M * kB + n_up];
  h->count[1] = (int64_t)C[M * kB + n_dn];
  int rc = HUB_OK;
  if (!dev_alloc((void **)&h->binom, sizeof(uint64_t) * kB * kB, "binomial table")) rc = HUB_ERR_OOM;
  if (rc == HUB_OK) {
    cudaError_t e = cudaMemcpy(h->binom, C.data(), sizeof(uint64_t) * kB * kB, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) rc = cuda_fail(e, "binomial upload", __FILE__, __LINE__);
  }
  for (int s = 0; s < 2 && rc == HUB_OK; ++s) {
    if (s == 1 && h->shared) {
      h->basis[1] = h->basis[0];
      break;
    }
    if (!dev_alloc((void **)&h->basis[s], sizeof(uint32_t) * h->count[s], "spin basis")) {
      rc = HUB_ERR_OOM;
      break;
    }
    k_unrank<<<grid_for(h->count[s], 256), 256>>>(M, h->N[s], h->count[s], h->binom, h->basis[s]);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = cuda_fail(e, "basis unrank", __FILE__, __LINE__);
  }
  if (rc != HUB_OK) {
    std::string msg = g_err;
    hub_free(h);
    g_err = msg;
    return rc;
  }
  *out = h;
  return HUB_OK;
}

extern "C" int hub_dims(hub_t h, int64_t *n_up, int64_t *n_dn) {
  if (!h) return fail(HUB_ERR_ARG, "hub_dims: NULL handle");
  if (n_up) *n_up = h->count[0];
  if (n_dn) *n_dn = h->count[1];
  return HUB_OK;
}

extern "C" int hub_get_basis(hub_t h, int spin, uint32_t *basis_host) {
  if (!h || !basis_host || (spin != 0 && spin != 1)) return fail(HUB_ERR_ARG, "hub_get_basis: bad argument");
  HUB_CUDA(cudaMemcpy(basis_host, h->basis[spin], sizeof(uint32_t) * h->count[spin], cudaMemcpyDeviceToHost));
  return HUB_OK;
}

extern "C" int hub_hopping(hub_t h, int n_bonds, const int32_t *bonds_host, const double *t_host,
                           const double *eps_host) {
  if (!h) return fail(HUB_ERR_ARG, "hub_hopping: NULL handle");
  if (n_bonds < 0 || n_bonds > kMaxBonds) return fail(HUB_ERR_ARG, "hub_hopping: need 0 <= n_bonds <= 255");
  if (n_bonds > 0 && (!bonds_host || !t_host)) return fail(HUB_ERR_ARG, "hub_hopping: NULL bonds or t");
  BondTable bt{};
  bt.n = n_bonds;
  for (int b = 0; b < n_bonds; ++b) {
    int i = bonds_host[2 * b], j = bonds_host[2 * b + 1];
    if (i < 0 || j < 0 || i >= h->M || j >= h->M || i == j)
      return fail(HUB_ERR_ARG, "hub_hopping: bond " + std::to_string(b) + " has a bad site");
    for (int c = 0; c < b; ++c) {
      int a0 = bonds_host[2 * c], a1 = bonds_host[2 * c + 1];
      if ((a0 == i && a1 == j) || (a0 == j && a1 == i))
        return fail(HUB_ERR_ARG, "hub_hopping: bond " + std::to_string(b) + " is listed twice");
    }
    if (!(t_host[b] == t_host[b]) || t_host[b] == INFINITY || t_host[b] == -INFINITY)
      return fail(HUB_ERR_ARG, "hub_hopping: t is not finite");
    bt.i[b] = (uint8_t)i;
    bt.j[b] = (uint8_t)j;
    bt.t[b] = t_host[b];
  }
  k0_leave(h);
  h->have_hop = false;
  h->n_bonds = n_bonds;
  h->bonds.assign(bonds_host, bonds_host + 2 * n_bonds);
  h->t.assign(t_host, t_host + n_bonds);
  h->eps.assign(h->M, 0.0);
  h->has_eps = false;
  if (eps_host)
    for (int i = 0; i < h->M; ++i) {
      h->eps[i] = eps_host[i];
      if (eps_host[i] != 0.0) h->has_eps = true;
    }
  for (int s = 0; s < 2; ++s) {
    if (s == 1 && h->shared) break;
    int rc = build_csr(h, s, bt);
    if (rc != HUB_OK) return rc;
  }
  for (int s = 0; s < 2; ++s) {
    dev_free(h->eps_state[s]);
    h->eps_state[s] = nullptr;
  }
  if (h->has_eps) {
    double *d_eps = nullptr;
    if (!dev_alloc((void **)&d_eps, sizeof(double) * h->M, "site energies")) return HUB_ERR_OOM;
    cudaError_t e = cudaMemcpy(d_eps, h->eps.data(), sizeof(double) * h->M, cudaMemcpyHostToDevice);
    for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
      if (s == 1 && h->shared) break;
      if (!dev_alloc((void **)&h->eps_state[s], sizeof(double) * h->count[s], "per-state site energy")) {
        dev_free(d_eps);
        return HUB_ERR_OOM;
      }
      k_eps_state<<<grid_for(h->count[s], 256), 256>>>(h->count[s], h->basis[s], h->M, d_eps, h->eps_state[s]);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    dev_free(d_eps);
    if (e != cudaSuccess) return cuda_fail(e, "site-energy tables", __FILE__, __LINE__);
  }
  h->have_hop = true;
  if (h->count[0] > 0 && h->count[1] > 0) {
    int rc = fast_build(h);
    if (rc != HUB_OK) {
      fast_release(h);
      return rc;
    }
  }
  return HUB_OK;
}

extern "C" int hub_set_U(hub_t h, int n_U, const double *U_host) {
  if (!h || !U_host) return fail(HUB_ERR_ARG, "hub_set_U: NULL argument");
  if (n_U != 1 && n_U != h->M) return fail(HUB_ERR_ARG, "hub_set_U: n_U must be 1 or M");
  h->U.assign(h->M, U_host[0]);
  bool uni = true;
  for (int i = 0; i < n_U; ++i) {
    if (!(U_host[i] == U_host[i])) return fail(HUB_ERR_ARG, "hub_set_U: U is NaN");
    h->U[i] = U_host[i];
    if (U_host[i] != U_host[0]) uni = false;
  }
  k0_leave(h);
  h->uniform_U = uni;
  h->U0 = U_host[0];
  h->have_U = true;
  return HUB_OK;
}

extern "C" int hub_csr_info(hub_t h, int spin, int64_t *nnz, int32_t *max_row) {
  if (!h || (spin != 0 && spin != 1)) return fail(HUB_ERR_ARG, "hub_csr_info: bad argument");
  if (!h->have_hop) return fail(HUB_ERR_STATE, "hub_csr_info: call hub_hopping first");
  const SpinCSR &c = h->csr[h->shared ? 0 : spin];
  if (nnz) *nnz = c.nnz;
  if (max_row) *max_row = c.max_row;
  return HUB_OK;
}

extern "C" int hub_get_csr(hub_t h, int spin, int32_t *rowptr_host, int32_t *cols_host, double *vals_host) {
  if (!h || (spin != 0 && spin != 1)) return fail(HUB_ERR_ARG, "hub_get_csr: bad argument");
  if (!h->have_hop) return fail(HUB_ERR_STATE, "hub_get_csr: call hub_hopping first");
  const SpinCSR &c = h->csr[h->shared ? 0 : spin];
  if (rowptr_host)
    HUB_CUDA(cudaMemcpy(rowptr_host, c.rowptr, sizeof(int32_t) * (h->count[spin] + 1), cudaMemcpyDeviceToHost));
  if (cols_host && c.nnz)
    HUB_CUDA(cudaMemcpy(cols_host, c.col, sizeof(int32_t) * c.nnz, cudaMemcpyDeviceToHost));
  if (vals_host && c.nnz)
    HUB_CUDA(cudaMemcpy(vals_host, c.val, sizeof(double) * c.nnz, cudaMemcpyDeviceToHost));
  return HUB_OK;
}

extern "C" void hub_free(hub_t h) {
  if (!h) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  dev_free(h->binom);
  dev_free(h->basis[0]);
  if (!h->shared) dev_free(h->basis[1]);
  for (int s = 0; s < 2; ++s) {
    if (s == 1 && h->shared) break;
    free_csr(h->csr[s]);
    dev_free(h->eps_state[s]);
  }
  for (int k = 0; k < 3; ++k) dev_free(h->work[k]);
  dev_free(h->psi_tmp);
  dev_free(h->ladder_map);
  dev_free(h->d_scal);
  dev_free(h->partials);
  if (h->h_scal) cudaFreeHost(h->h_scal);
  dev_free(h->hx);
  dev_free(h->hy);
  dev_free(h->hx2);
  dev_free(h->hy2);
  fast_release(h);
  k0_release(h);
  small_release(h);
  for (int k = 0; k < hub_ctx::kProfKinds; ++k) {
    for (cudaEvent_t e : h->ev_start[k]) cudaEventDestroy(e);
    for (cudaEvent_t e : h->ev_end[k]) cudaEventDestroy(e);
  }
  cudaSetDevice(prev);
  delete h;
}
