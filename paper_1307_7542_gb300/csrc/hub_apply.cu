// hub_apply.cu -- the matrix-free Hamiltonian product (K3).
//
// Sec. IV.A, Eq. 11: H = I_dn (x) H_up + H_dn (x) I_up + H_U.  With the state stored as
// the count_dn x count_up row-major matrix X (Eq. count2; the vecold reshape of Sec.
// IV.A), the spin-up term is X H_up^T -- a gather inside one row of X -- and the
// spin-down term is H_dn X -- a combination of whole rows of X (Sec. IV.A: "vecnew =
// H_up x vecold" and "vecnew = vecold x H_dn^T", transposed to this row-major layout).
// The diagonal (Sec. III.B) is sum_i U_i bit_i(I_up & I_dn) + eps(I_up) + eps(I_dn),
// computed on the fly from popcount instead of Algorithm II's index_U tables.
//
// Kernel shape (FP64 path): one CTA per row d of X (grid-stride).  The CTA stages row d
// in shared memory when it fits; each thread owns columns u and sums the H_up row of u
// (gather from shared memory) and the H_dn row of d (coalesced loads of the neighbour
// rows X[d'][u], served from L2).
#include "hub_internal.cuh"

namespace hub {

// gate: null, or a device flag; the kernel does nothing while gate[0] is 0 (the fast path
// passes its out-of-window flag, so that this kernel multiplies exactly the vectors the
// double-float kernels cannot).
template <bool kStage>
__global__ void __launch_bounds__(512) k_apply_f64(const Ham H, const double *__restrict__ x,
                                                   double *__restrict__ y, const int *__restrict__ gate) {
  if (gate && gate[0] == 0) return;
  extern __shared__ double xs[];
  const int64_t nu = H.n_up, nd = H.n_dn;
  for (int64_t d = blockIdx.x; d < nd; d += gridDim.x) {
    const double *__restrict__ xrow = x + d * nu;
    if (kStage) {
      for (int64_t u = threadIdx.x; u < nu; u += blockDim.x) xs[u] = xrow[u];
      __syncthreads();
    }
    const uint32_t Id = H.basis_dn[d];
    const int32_t k0 = H.rp_dn[d], k1 = H.rp_dn[d + 1];
    for (int64_t u = threadIdx.x; u < nu; u += blockDim.x) {
      const double xv = kStage ? xs[u] : xrow[u];
      double acc = diag_of(H, H.basis_up[u], Id, u, d) * xv;
      const int32_t j0 = H.rp_up[u], j1 = H.rp_up[u + 1];
      for (int32_t k = j0; k < j1; ++k) {
        const int32_t c = H.col_up[k];
        acc = fma(H.val_up[k], kStage ? xs[c] : xrow[c], acc);
      }
      for (int32_t k = k0; k < k1; ++k) acc = fma(H.val_dn[k], x[(int64_t)H.col_dn[k] * nu + u], acc);
      y[d * nu + u] = acc;
    }
    if (kStage) __syncthreads();
  }
}

static size_t stage_bytes(const Ham &H) { return sizeof(double) * (size_t)H.n_up; }

static int apply_kernels(hub_ctx *h, const double *x, double *y, cudaStream_t s);

constexpr int64_t kMaxTimed = 65536;

int prof_mark(hub_ctx *h, int kind, bool begin, cudaStream_t s) {
  if (!h->prof) return HUB_OK;
  int64_t &nt = h->n_timed[kind];
  if (begin) {
    if (nt >= kMaxTimed) return HUB_OK;
    if ((int64_t)h->ev_start[kind].size() <= nt) {
      cudaEvent_t e0, e1;
      HUB_CUDA(cudaEventCreate(&e0));
      HUB_CUDA(cudaEventCreate(&e1));
      h->ev_start[kind].push_back(e0);
      h->ev_end[kind].push_back(e1);
    }
    HUB_CUDA(cudaEventRecord(h->ev_start[kind][nt], s));
  } else {
    ++h->n_launch[kind];
    if (nt >= kMaxTimed) return HUB_OK;
    HUB_CUDA(cudaEventRecord(h->ev_end[kind][nt], s));
    ++nt;
  }
  return HUB_OK;
}

int apply_launch(hub_ctx *h, const double *x, double *y, cudaStream_t s) {
  int rc = prof_mark(h, HUB_PROF_APPLY, true, s);
  if (rc) return rc;
  if ((rc = apply_kernels(h, x, y, s))) return rc;
  return prof_mark(h, HUB_PROF_APPLY, false, s);
}

static int apply_kernels(hub_ctx *h, const double *x, double *y, cudaStream_t s) {
  const Ham H = h->view();
  if (H.n_up == 0 || H.n_dn == 0) return HUB_OK;
  if (h->k0) return k0_apply(h, x, y, s);
  if (use_fast(h)) return fast_apply_f64(h, x, y, s);
  return f64_apply(h, x, y, nullptr, s);
}

int f64_apply(hub_ctx *h, const double *x, double *y, const int *gate, cudaStream_t s) {
  const Ham H = h->view();
  count_launch(h);
  const size_t smem = stage_bytes(H);
  const int threads = H.n_up >= 512 ? 512 : (H.n_up >= 128 ? 256 : 64);
  int64_t grid = H.n_dn;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (grid > cap) grid = cap;
  if (smem <= 200 * 1024) {
    HUB_CUDA(cudaFuncSetAttribute(k_apply_f64<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    k_apply_f64<true><<<(int)grid, threads, smem, s>>>(H, x, y, gate);
  } else {
    k_apply_f64<false><<<(int)grid, threads, 0, s>>>(H, x, y, gate);
  }
  HUB_LAUNCH_CHECK();
  return HUB_OK;
}

static int check_ready(const hub_ctx *h, const char *who) {
  if (!h) return fail(HUB_ERR_ARG, std::string(who) + ": NULL handle");
  if (!h->have_hop) return fail(HUB_ERR_STATE, std::string(who) + ": call hub_hopping first");
  if (!h->have_U) return fail(HUB_ERR_STATE, std::string(who) + ": call hub_set_U first");
  return HUB_OK;
}

int ready(const hub_ctx *h, const char *who) { return check_ready(h, who); }

}  // namespace hub

using namespace hub;

extern "C" int hub_apply(hub_t h, const double *x_dev, double *y_dev, void *stream) {
  int rc = check_ready(h, "hub_apply");
  if (rc) return rc;
  if (!x_dev || !y_dev) return fail(HUB_ERR_ARG, "hub_apply: NULL vector");
  const int64_t D = vec_len(h);
  if (x_dev < y_dev + D && y_dev < x_dev + D) return fail(HUB_ERR_ARG, "hub_apply: x and y overlap");
  return apply_launch(h, x_dev, y_dev, (cudaStream_t)stream);
}

// The FP64 device input and output vector of a host-buffer apply (x, y: hx and hy, or the
// second pair hx2 and hy2), allocated on first use.
static int host_apply_buffers(hub_ctx *h, double **x, double **y) {
  if (*x) return HUB_OK;
  const int64_t D = vec_len(h);
  if (!dev_alloc((void **)x, sizeof(double) * D, "host-apply input") ||
      !dev_alloc((void **)y, sizeof(double) * D, "host-apply output")) {
    dev_free(*x);
    *x = nullptr;
    return HUB_ERR_OOM;
  }
  return HUB_OK;
}

extern "C" int hub_apply_host(hub_t h, const double *x_host, double *y_host, void *stream) {
  int rc = check_ready(h, "hub_apply_host");
  if (rc) return rc;
  if (!x_host || !y_host) return fail(HUB_ERR_ARG, "hub_apply_host: NULL vector");
  const int64_t D = vec_len(h);
  if ((rc = host_apply_buffers(h, &h->hx, &h->hy))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (use_fast(h)) return fast_apply_host(h, x_host, y_host, h->hx, h->hy, s);
  HUB_CUDA(cudaMemcpyAsync(h->hx, x_host, sizeof(double) * D, cudaMemcpyHostToDevice, s));
  rc = apply_launch(h, h->hx, h->hy, s);
  if (rc) return rc;
  HUB_CUDA(cudaMemcpyAsync(y_host, h->hy, sizeof(double) * D, cudaMemcpyDeviceToHost, s));
  HUB_CUDA(cudaStreamSynchronize(s));
  return HUB_OK;
}

extern "C" int hub_apply_host_many(hub_t h, int64_t n_vec, const double *x_host, double *y_host, void *stream) {
  int rc = check_ready(h, "hub_apply_host_many");
  if (rc) return rc;
  if (n_vec < 0) return fail(HUB_ERR_ARG, "hub_apply_host_many: negative vector count");
  if (n_vec == 0) return HUB_OK;
  if (!x_host || !y_host) return fail(HUB_ERR_ARG, "hub_apply_host_many: NULL vector");
  const int64_t D = vec_len(h);
  if (D > 0 && n_vec > (int64_t)(SIZE_MAX / sizeof(double)) / D)
    return fail(HUB_ERR_ARG, "hub_apply_host_many: vector count too large");
  const uintptr_t xa = (uintptr_t)x_host, ya = (uintptr_t)y_host, bytes = (uintptr_t)(n_vec * D) * sizeof(double);
  if (xa != ya && xa < ya + bytes && ya < xa + bytes)
    return fail(HUB_ERR_ARG, "hub_apply_host_many: x and y overlap without being the same array");
  if (n_vec == 1 || !use_fast(h) || !fast_host_pipelined(h)) {   // one call per vector
    for (int64_t v = 0; v < n_vec; ++v)
      if ((rc = hub_apply_host(h, x_host + v * D, y_host + v * D, stream))) return rc;
    return HUB_OK;
  }
  if ((rc = host_apply_buffers(h, &h->hx, &h->hy)) || (rc = host_apply_buffers(h, &h->hx2, &h->hy2))) return rc;
  double *const xd[2] = {h->hx, h->hx2}, *const yd[2] = {h->hy, h->hy2};
  return fast_apply_host_many(h, n_vec, x_host, y_host, xd, yd, (cudaStream_t)stream);
}

extern "C" int hub_profile(hub_t h, int enable) {
  if (!h) return fail(HUB_ERR_ARG, "hub_profile: NULL handle");
  h->prof = enable != 0;
  if (h->prof) {
    for (int k = 0; k < hub_ctx::kProfKinds; ++k) h->n_launch[k] = h->n_timed[k] = 0;
    h->n_kernels = 0;
  }
  return HUB_OK;
}

extern "C" int hub_profile_read(hub_t h, int kind, double *ms, int64_t *launches, int64_t *kernel_launches) {
  if (!h || kind < 0 || kind >= hub_ctx::kProfKinds) return fail(HUB_ERR_ARG, "hub_profile_read: bad argument");
  double total = 0.0;
  for (int64_t k = 0; k < h->n_timed[kind]; ++k) {
    HUB_CUDA(cudaEventSynchronize(h->ev_end[kind][k]));
    float t = 0.f;
    HUB_CUDA(cudaEventElapsedTime(&t, h->ev_start[kind][k], h->ev_end[kind][k]));
    total += t;
  }
  const int64_t nt = h->n_timed[kind], nl = h->n_launch[kind];
  if (ms) *ms = nt ? total * (double)nl / (double)nt : 0.0;
  if (launches) *launches = nl;
  if (kernel_launches) *kernel_launches = h->n_kernels;
  return HUB_OK;
}

extern "C" int hub_set_mode(hub_t h, int mode) {
  if (!h || (mode != HUB_MODE_AUTO && mode != HUB_MODE_FP64)) return fail(HUB_ERR_ARG, "hub_set_mode: bad argument");
  h->mode = mode;
  return HUB_OK;
}

extern "C" int hub_test_fail_waits(hub_t h, int enable) {
  if (!h) return fail(HUB_ERR_ARG, "hub_test_fail_waits: NULL handle");
  h->fail_waits = enable != 0;
  return HUB_OK;
}

extern "C" int hub_check(hub_t h) {
  if (!h) return fail(HUB_ERR_ARG, "hub_check: NULL handle");
  HUB_CUDA(cudaDeviceSynchronize());
  const int rc = fast_check_error(h);
  return rc ? rc : small_check_error(h);
}
