// hub_green.cu -- one-particle Green's function at zero temperature (Sec. VII, Eq. count8).
//
// G_sigma(p, z) = <psi0| c_p (z + E0 - H)^-1 c+_p |psi0> + <psi0| c+_p (z - E0 + H)^-1 c_p |psi0>
// is evaluated as two continued fractions (Sec. VII): the Lanczos recurrence of Sec. IV / V
// started from v = c+_p psi0 (sector N_sigma + 1) or v = c_p psi0 (sector N_sigma - 1) gives
// the tridiagonal T of H in the Krylov space of v, and <v|(z -/+ (H - E0))^-1|v> is the
// (0, 0) element of the resolvent of T, a continued fraction in its alpha_j and beta_j.
//
// hub_ladder forms v as in the vecin construction of Sec. VII: a state of the target sector
// whose site p (spin sigma) is occupied (c+) or empty (c) comes from exactly one state of the
// source sector, the target state with that bit flipped, found by its combinadic rank; the
// sign is the Jordan-Wigner sign of the operator order of Sec. II, Eq. 7 (all up operators
// before all down operators, ascending sites).  For spin up the map acts on columns of the
// count_dn x count_up state matrix (a signed gather inside every row), for spin down on rows
// (signed copies of whole rows).
#include <algorithm>
#include <cmath>
#include <complex>
#include <string>

#include "hub_internal.cuh"

namespace hub {

int ready(const hub_ctx *h, const char *who);

constexpr int32_t kNoSource = INT32_MIN;   // target state outside the image of the operator

// map[r] for target state r (basis `to`): rank of its source state s (sign +), ~rank (sign -)
// or kNoSource.  bit = 1 << site; s = target ^ bit, required to have the bit set (c) or clear
// (c+); sign = (-1)^(parity0 + set bits of s below the site).
__global__ void k_ladder_map(int64_t n, const uint32_t *__restrict__ basis_to, uint32_t bit, int create,
                             int parity0, const uint64_t *__restrict__ C, int32_t *__restrict__ map) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t t = basis_to[r];
    const bool occupied = (t & bit) != 0;
    if (occupied != (create != 0)) {
      map[r] = kNoSource;
      continue;
    }
    const uint32_t s = t ^ bit;
    const int neg = (__popc(s & (bit - 1u)) + parity0) & 1;
    const int32_t idx = (int32_t)rank_of(s, C);
    map[r] = neg ? ~idx : idx;
  }
}

__device__ __forceinline__ double mapped(int32_t m, const double *__restrict__ src) {
  return m == kNoSource ? 0.0 : (m >= 0 ? src[m] : -src[~m]);
}

// spin up: y[d][r] = sign_r x[d][src_r] (one row per block and step; the gathers of a row
// are served from L1, the stores are coalesced)
__global__ void k_ladder_cols(int64_t rows, int64_t n_from, int64_t n_to, const int32_t *__restrict__ map,
                              const double *__restrict__ x, double *__restrict__ y) {
  for (int64_t d = blockIdx.x; d < rows; d += gridDim.x)
    for (int64_t r = threadIdx.x; r < n_to; r += blockDim.x) y[d * n_to + r] = mapped(map[r], x + d * n_from);
}

// spin down: y[r][u] = sign_r x[src_r][u] (whole rows)
__global__ void k_ladder_rows(int64_t n_to, int64_t cols, const int32_t *__restrict__ map,
                              const double *__restrict__ x, double *__restrict__ y) {
  for (int64_t r = blockIdx.x; r < n_to; r += gridDim.x) {
    const int32_t m = map[r];
    const double *src = m == kNoSource ? nullptr : x + (int64_t)(m >= 0 ? m : ~m) * cols;
    const double sg = m >= 0 ? 1.0 : -1.0;
    for (int64_t u = threadIdx.x; u < cols; u += blockDim.x) y[r * cols + u] = src ? sg * src[u] : 0.0;
  }
}

}  // namespace hub

using namespace hub;

extern "C" int hub_ladder(hub_t from, hub_t to, int site, int spin, int create, const double *x_dev,
                          double *y_dev, void *stream) {
  if (!from || !to) return fail(HUB_ERR_ARG, "hub_ladder: NULL handle");
  if (from->M != to->M) return fail(HUB_ERR_ARG, "hub_ladder: the two handles have different M");
  if (from->k0 || to->k0) return fail(HUB_ERR_STATE, "hub_ladder: not available in the k = 0 sector (hub_set_symmetry)");
  if (site < 0 || site >= from->M) return fail(HUB_ERR_ARG, "hub_ladder: site out of range");
  if (spin != HUB_SPIN_UP && spin != HUB_SPIN_DN) return fail(HUB_ERR_ARG, "hub_ladder: bad spin");
  if (!x_dev || !y_dev) return fail(HUB_ERR_ARG, "hub_ladder: NULL vector");
  const int o = 1 - spin;
  const int dN = create ? 1 : -1;
  if (to->N[spin] != from->N[spin] + dN || to->N[o] != from->N[o])
    return fail(HUB_ERR_ARG, "hub_ladder: target sector must differ by one electron of the given spin");
  if (from->device != to->device) return fail(HUB_ERR_ARG, "hub_ladder: handles on different devices");
  const int64_t D_from = from->count[0] * from->count[1], D_to = to->count[0] * to->count[1];
  if (x_dev < y_dev + D_to && y_dev < x_dev + D_from) return fail(HUB_ERR_ARG, "hub_ladder: x and y overlap");
  const int64_t n_map = to->count[spin];
  if (n_map > to->ladder_cap) {
    dev_free(to->ladder_map);
    to->ladder_map = nullptr;
    to->ladder_cap = 0;
    if (!dev_alloc((void **)&to->ladder_map, sizeof(int32_t) * n_map, "ladder map")) return HUB_ERR_OOM;
    to->ladder_cap = n_map;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // a down-spin operator passes all N_up up operators first (Sec. II, Eq. 7)
  const int parity0 = spin == HUB_SPIN_DN ? (from->N[HUB_SPIN_UP] & 1) : 0;
  const int sms = num_sms();
  k_ladder_map<<<(int)std::min<int64_t>((n_map + 255) / 256, (int64_t)sms * 8), 256, 0, s>>>(
      n_map, to->basis[spin], 1u << site, create, parity0, from->binom, to->ladder_map);
  HUB_LAUNCH_CHECK();
  if (D_to == 0) return HUB_OK;
  if (spin == HUB_SPIN_UP) {
    const int64_t rows = to->count[1];
    k_ladder_cols<<<(int)std::min<int64_t>(rows, (int64_t)sms * 8), 256, 0, s>>>(rows, from->count[0], to->count[0],
                                                                                   to->ladder_map, x_dev, y_dev);
  } else {
    const int64_t rows = to->count[1];
    k_ladder_rows<<<(int)std::min<int64_t>(rows, (int64_t)sms * 8), 256, 0, s>>>(rows, to->count[0], to->ladder_map,
                                                                                   x_dev, y_dev);
  }
  HUB_LAUNCH_CHECK();
  return HUB_OK;
}

extern "C" int hub_green_coeffs(hub_t h, const double *v_dev, int k, double *alpha_host, double *beta_host,
                                double *norm2_host, int *k_out, void *stream) {
  int rc = ready(h, "hub_green_coeffs");
  if (rc) return rc;
  if (!v_dev || !alpha_host || !beta_host || !norm2_host || !k_out || k < 1)
    return fail(HUB_ERR_ARG, "hub_green_coeffs: bad argument");
  double E0 = 0.0;
  int it = 0;
  h->start_norm = -1.0;
  rc = hub_lanczos_ground(h, v_dev, k, 0.0, &E0, nullptr, &it, stream);
  if (rc == HUB_ERR_ARG && h->start_norm == 0.0) {   // v = 0: the operator annihilates psi0
    *norm2_host = 0.0;
    *k_out = 0;
    return HUB_OK;
  }
  if (rc < 0) return rc;
  for (int j = 0; j < it; ++j) {
    alpha_host[j] = h->alpha[j];
    beta_host[j] = j < (int)h->beta.size() ? h->beta[j] : 0.0;
  }
  *norm2_host = h->start_norm * h->start_norm;
  *k_out = it;
  return HUB_OK;
}

extern "C" int hub_green_eval(int k, const double *alpha, const double *beta, double norm2, double E0, int sign,
                              int n_z, const double *z_re, const double *z_im, double *g_re, double *g_im) {
  if (k < 0 || n_z < 0 || (sign != 1 && sign != -1) || (k > 0 && (!alpha || !beta)) ||
      (n_z > 0 && (!z_re || !z_im || !g_re || !g_im)))
    return fail(HUB_ERR_ARG, "hub_green_eval: bad argument");
  for (int i = 0; i < n_z; ++i) {
    const std::complex<double> z(z_re[i], z_im[i]);
    std::complex<double> g(0.0, 0.0);
    if (k > 0) {
      // resolvent of T, bottom up: f_j = z - s (alpha_j - E0) - beta_j^2 / f_{j+1}
      std::complex<double> f = z - (double)sign * (alpha[k - 1] - E0);
      for (int j = k - 2; j >= 0; --j) f = z - (double)sign * (alpha[j] - E0) - beta[j] * beta[j] / f;
      g = norm2 / f;
    }
    g_re[i] = g.real();
    g_im[i] = g.imag();
  }
  return HUB_OK;
}
