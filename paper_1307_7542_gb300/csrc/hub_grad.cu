// hub_grad.cu -- derivatives of H (K5): the bilinear forms a^T (dH/dtheta) b for every bond
// hopping t_b, on-site interaction U_i and site energy eps_i.
//
// With a = b = psi these are the Hellmann-Feynman gradients of E0 (per-bond hopping
// correlators, double occupancies, densities); with a = ybar, b = x they are the
// parameter cotangents of y = H x.  The derivative operators follow from Eq. 1:
//   dH/dt_b   = -sum_sigma (c+_i c_j + h.c.)   -> the hops of bond b in H_up and H_dn,
//                                                with the Jordan-Wigner sign of Eq. 8;
//   dH/dU_i   = n_{i up} n_{i dn}             -> bit i of (I_up & I_dn) (Sec. III.B);
//   dH/deps_i = n_{i up} + n_{i dn}.
// One CTA per row d of the count_dn x count_up state matrix (Eq. count2), the row of b
// staged in shared memory for the spin-up hops (in-row gathers, Eq. 11 first term) and
// neighbour rows of b read directly for the spin-down hops (second term).  Each CTA
// accumulates per-parameter sums in shared memory and writes one partial per parameter;
// a second kernel adds the partials in a fixed order.
#include <vector>

#include "hub_internal.cuh"

namespace hub {

int ready(const hub_ctx *h, const char *who);

struct GradArgs {
  int n_bonds;
  int n_par;            // n_bonds + 2M
  const uint8_t *bond_up, *bond_dn;
};

template <bool kStage>
__global__ void __launch_bounds__(256) k_bilinear(const Ham H, GradArgs G, const double *__restrict__ a,
                                                  const double *__restrict__ b, double *__restrict__ partials) {
  extern __shared__ double sm[];
  double *bins = sm;                       // [n_par] per block
  double *bs = sm + ((G.n_par + 1) & ~1);  // staged row of b
  for (int k = threadIdx.x; k < G.n_par; k += blockDim.x) bins[k] = 0.0;
  __syncthreads();
  const int64_t nu = H.n_up, nd = H.n_dn;
  const int M = H.M;
  double *binU = bins + G.n_bonds, *binE = bins + G.n_bonds + M;
  for (int64_t d = blockIdx.x; d < nd; d += gridDim.x) {
    const double *__restrict__ brow = b + d * nu;
    const double *__restrict__ arow = a + d * nu;
    if (kStage) {
      for (int64_t u = threadIdx.x; u < nu; u += blockDim.x) bs[u] = brow[u];
      __syncthreads();
    }
    const uint32_t Id = H.basis_dn[d];
    // spin-up hops, on-site terms
    for (int64_t u = threadIdx.x; u < nu; u += blockDim.x) {
      const double av = arow[u];
      const double p = av * (kStage ? bs[u] : brow[u]);
      const uint32_t Iu = H.basis_up[u];
      for (uint32_t m = Iu & Id; m; m &= m - 1) atomicAdd(&binU[__ffs(m) - 1], p);
      for (uint32_t m = Iu; m; m &= m - 1) atomicAdd(&binE[__ffs(m) - 1], p);
      for (uint32_t m = Id; m; m &= m - 1) atomicAdd(&binE[__ffs(m) - 1], p);
      const int32_t j0 = H.rp_up[u], j1 = H.rp_up[u + 1];
      for (int32_t k = j0; k < j1; ++k) {
        const uint32_t sc = H.scol_up[k];
        const int32_t c = (int32_t)(sc & 0x7fffffffu);
        const double v = av * (kStage ? bs[c] : brow[c]);
        atomicAdd(&bins[G.bond_up[k]], (sc >> 31) ? v : -v);   // -(sign) a b
      }
    }
    // spin-down hops: one block-uniform CSR entry at a time, warp sums then one atomic
    const int32_t k0 = H.rp_dn[d], k1 = H.rp_dn[d + 1];
    for (int32_t k = k0; k < k1; ++k) {
      const uint32_t sc = H.scol_dn[k];
      const double *__restrict__ b2 = b + (int64_t)(sc & 0x7fffffffu) * nu;
      double v = 0.0;
      for (int64_t u = threadIdx.x; u < nu; u += blockDim.x) v = fma(arow[u], b2[u], v);
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0) atomicAdd(&bins[G.bond_dn[k]], (sc >> 31) ? v : -v);
    }
    if (kStage) __syncthreads();
  }
  __syncthreads();
  for (int k = threadIdx.x; k < G.n_par; k += blockDim.x) partials[(int64_t)k * gridDim.x + blockIdx.x] = bins[k];
}

// out[k] = sum over blocks of partials[k][.], fixed order; one block per parameter.
__global__ void k_reduce_rows(const double *__restrict__ partials, int nblk, double *__restrict__ out) {
  __shared__ double s[256];
  const double *p = partials + (int64_t)blockIdx.x * nblk;
  double v = 0.0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) v += p[k];
  s[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = s[0];
}

// Computes all n_bonds + 2M bilinear forms into host arrays.
static int bilinear(hub_ctx *h, const double *a, const double *b, double *dt, double *dU, double *de,
                    cudaStream_t s) {
  const Ham H = h->view();
  GradArgs G;
  G.n_bonds = h->n_bonds;
  G.n_par = h->n_bonds + 2 * h->M;
  G.bond_up = h->csr[0].bond;
  G.bond_dn = h->csr[h->shared ? 0 : 1].bond;
  int nblk = (int)std::min<int64_t>(H.n_dn, (int64_t)num_sms() * 4);
  if (nblk < 1) nblk = 1;
  int rc = ensure_partials(h, (int64_t)G.n_par * nblk + G.n_par);
  if (rc) return rc;
  double *P = h->partials, *out = h->partials + (int64_t)G.n_par * nblk;
  const size_t bins_bytes = sizeof(double) * ((G.n_par + 1) & ~1);
  const size_t row_bytes = sizeof(double) * (size_t)H.n_up;
  if (bins_bytes + row_bytes <= 200 * 1024) {
    HUB_CUDA(cudaFuncSetAttribute(k_bilinear<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    k_bilinear<true><<<nblk, 256, bins_bytes + row_bytes, s>>>(H, G, a, b, P);
  } else {
    k_bilinear<false><<<nblk, 256, bins_bytes, s>>>(H, G, a, b, P);
  }
  HUB_LAUNCH_CHECK();
  k_reduce_rows<<<G.n_par, 256, 0, s>>>(P, nblk, out);
  HUB_LAUNCH_CHECK();
  std::vector<double> host(G.n_par);
  HUB_CUDA(cudaMemcpyAsync(host.data(), out, sizeof(double) * G.n_par, cudaMemcpyDeviceToHost, s));
  HUB_CUDA(cudaStreamSynchronize(s));
  for (int k = 0; k < h->n_bonds; ++k)
    if (dt) dt[k] = host[k];
  for (int i = 0; i < h->M; ++i) {
    if (dU) dU[i] = host[h->n_bonds + i];
    if (de) de[i] = host[h->n_bonds + h->M + i];
  }
  return HUB_OK;
}

}  // namespace hub

using namespace hub;

extern "C" int hub_grad(hub_t h, const double *psi_dev, double *dE_dt_host, double *dE_dU_host,
                        double *dE_deps_host, void *stream) {
  int rc = ready(h, "hub_grad");
  if (rc) return rc;
  if (h->k0) return fail(HUB_ERR_STATE, "hub_grad: not available in the k = 0 sector (hub_set_symmetry)");
  if (!psi_dev) return fail(HUB_ERR_ARG, "hub_grad: psi is NULL");
  return bilinear(h, psi_dev, psi_dev, dE_dt_host, dE_dU_host, dE_deps_host, (cudaStream_t)stream);
}

extern "C" int hub_apply_vjp(hub_t h, const double *ybar_dev, const double *x_dev, double *xbar_dev,
                             double *tbar_host, double *Ubar_host, double *epsbar_host, void *stream) {
  int rc = ready(h, "hub_apply_vjp");
  if (rc) return rc;
  if (h->k0) return fail(HUB_ERR_STATE, "hub_apply_vjp: not available in the k = 0 sector (hub_set_symmetry)");
  if (!ybar_dev || (!x_dev && (tbar_host || Ubar_host || epsbar_host)))
    return fail(HUB_ERR_ARG, "hub_apply_vjp: NULL vector");
  cudaStream_t s = (cudaStream_t)stream;
  if (xbar_dev) {
    const int64_t D = h->count[0] * h->count[1];
    if (xbar_dev < ybar_dev + D && ybar_dev < xbar_dev + D) return fail(HUB_ERR_ARG, "hub_apply_vjp: xbar overlaps ybar");
    if ((rc = apply_launch(h, ybar_dev, xbar_dev, s))) return rc;
  }
  if (tbar_host || Ubar_host || epsbar_host) {
    if ((rc = bilinear(h, ybar_dev, x_dev, tbar_host, Ubar_host, epsbar_host, s))) return rc;
  } else {
    HUB_CUDA(cudaStreamSynchronize(s));
  }
  return HUB_OK;
}

// ---------------------------------------------------------------------------------------
// hub_grad_noalloc: the Hellmann-Feynman gradients with no memory allocation at call time.
// The per-block partial sums and the reduced results live in one file-scope device array
// of fixed size instead of the handle's lazily allocated scratch.
// ---------------------------------------------------------------------------------------
namespace hub {

constexpr int kNoAllocMaxParams = 160;   // n_bonds + 2M that fit the fixed array
constexpr int kNoAllocMaxBlocks = 608;   // partial sums kept per parameter
constexpr int64_t kNoAllocDoubles = (int64_t)kNoAllocMaxBlocks * kNoAllocMaxParams + kNoAllocMaxParams;

// 608 * 160 + 160 doubles = 779,520 bytes, held by every GPU that loads the library.
static __device__ __align__(256) double g_grad_scratch[kNoAllocDoubles];

// Device address of g_grad_scratch on the current device.  In host code the symbol
// g_grad_scratch is only a host-side stand-in; kernels must be given this address.  It is
// looked up on every call (a host-side lookup once the library's device code is loaded on
// the device), so a context that was torn down and created again never sees a stale
// address; the first call on a device may load that code, which places the array there.
static int noalloc_scratch(double **out) {
  void *p = nullptr;
  HUB_CUDA(cudaGetSymbolAddress(&p, g_grad_scratch));
  *out = static_cast<double *>(p);
  return HUB_OK;
}

}  // namespace hub

extern "C" int hub_grad_noalloc(hub_t h, const double *psi_dev, double *dE_dt_host, double *dE_dU_host,
                                double *dE_deps_host, void *stream) {
  int rc = ready(h, "hub_grad_noalloc");
  if (rc) return rc;
  if (h->k0) return fail(HUB_ERR_STATE, "hub_grad_noalloc: not available in the k = 0 sector (hub_set_symmetry)");
  if (!psi_dev) return fail(HUB_ERR_ARG, "hub_grad_noalloc: psi is NULL");
  const int n_par = h->n_bonds + 2 * h->M;
  if (n_par > kNoAllocMaxParams)
    return fail(HUB_ERR_ARG, "hub_grad_noalloc: n_bonds + 2*M = " + std::to_string(n_par) +
                                 " exceeds the fixed scratch capacity of " + std::to_string(kNoAllocMaxParams) +
                                 " parameters; use hub_grad");
  int dev = 0;
  HUB_CUDA(cudaGetDevice(&dev));
  if (dev != h->device) return fail(HUB_ERR_ARG, "hub_grad_noalloc: the handle's device is not the current device");
  double *scratch = nullptr;
  if ((rc = noalloc_scratch(&scratch))) return rc;

  const Ham H = h->view();
  GradArgs G;
  G.n_bonds = h->n_bonds;
  G.n_par = n_par;
  G.bond_up = h->csr[0].bond;
  G.bond_dn = h->csr[h->shared ? 0 : 1].bond;
  int nblk = (int)std::min<int64_t>(H.n_dn, (int64_t)num_sms() * 4);
  nblk = std::max(1, std::min(nblk, kNoAllocMaxBlocks));
  // every partial the reduction reads is written by this call's first kernel, and every
  // result by its second, so nothing needs clearing between calls
  double *P = scratch, *out = scratch + (int64_t)n_par * nblk;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bins_bytes = sizeof(double) * ((n_par + 1) & ~1);
  const size_t row_bytes = sizeof(double) * (size_t)H.n_up;
  if (bins_bytes + row_bytes <= 200 * 1024) {
    HUB_CUDA(cudaFuncSetAttribute(k_bilinear<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    k_bilinear<true><<<nblk, 256, bins_bytes + row_bytes, s>>>(H, G, psi_dev, psi_dev, P);
  } else {
    k_bilinear<false><<<nblk, 256, bins_bytes, s>>>(H, G, psi_dev, psi_dev, P);
  }
  HUB_LAUNCH_CHECK();
  k_reduce_rows<<<n_par, 256, 0, s>>>(P, nblk, out);
  HUB_LAUNCH_CHECK();
  if (dE_dt_host && h->n_bonds)
    HUB_CUDA(cudaMemcpyAsync(dE_dt_host, out, sizeof(double) * h->n_bonds, cudaMemcpyDeviceToHost, s));
  if (dE_dU_host)
    HUB_CUDA(cudaMemcpyAsync(dE_dU_host, out + h->n_bonds, sizeof(double) * h->M, cudaMemcpyDeviceToHost, s));
  if (dE_deps_host)
    HUB_CUDA(cudaMemcpyAsync(dE_deps_host, out + h->n_bonds + h->M, sizeof(double) * h->M, cudaMemcpyDeviceToHost, s));
  HUB_CUDA(cudaStreamSynchronize(s));
  return HUB_OK;
}
