// hub_block.cu -- block Lanczos: several start vectors at once, for low-lying levels with
// their multiplicities (Sec. IV: the Lanczos method needs only the product H q, here applied
// to a block of k vectors per step; a single start vector finds each degenerate level once).
//
// Block recurrence with full re-orthogonalisation (every block is kept on the device):
//   Q_1 R_0 = X_0                                  (orthonormal columns, Cholesky QR twice)
//   W = H Q_j - Q_{j-1} B_{j-1}^T,  A_j = Q_j^T W,  W -= Q_j A_j,
//   W -= Q_{<=j} (Q_{<=j}^T W)  (twice),  Q_{j+1} B_j = W   (Cholesky QR twice)
// T is the symmetric block-tridiagonal matrix of the A_j (diagonal) and B_j (below the
// diagonal); its eigenvalues are the Ritz values, each level of multiplicity g <= k found g
// times, and |H y - theta y| = |B_m s_m| with s_m the last block of T's eigenvector s.  The
// products are the library's own (fast or FP64 path, hub_apply's accuracy); the block
// vectors are FP64, column-contiguous (vector c of a block at c * D).
#include <algorithm>
#include <cmath>
#include <vector>

#include "hub_internal.cuh"

namespace hub {

int ready(const hub_ctx *h, const char *who);

namespace {

constexpr int kMaxBlock = 8;        // block size k
constexpr int kMaxKrylov = 512;     // k * steps (T is diagonalised densely on the host)
constexpr int kGramTile = 8;        // vectors of X per CTA of the Gram kernel
constexpr int kGramThreads = 256;

// Partial Gram products: for the X-tile t = blockIdx.y (vectors t*8 .. t*8+7 of X, at most
// nx) and the Q <= 8 vectors of Y, CTA blockIdx.x sums X_a[n] Y_b[n] over its grid-stride
// share of n; part[(t * gridDim.x + blockIdx.x) * 64 + (a % 8) * 8 + b].
template <int Q>
__global__ void __launch_bounds__(kGramThreads) k_gram_part(int64_t D, const double *__restrict__ X, int nx,
                                                            const double *__restrict__ Y,
                                                            double *__restrict__ part) {
  const int a0 = blockIdx.y * kGramTile;
  const int na = min(kGramTile, nx - a0);
  double acc[kGramTile][Q];
#pragma unroll
  for (int a = 0; a < kGramTile; ++a)
#pragma unroll
    for (int b = 0; b < Q; ++b) acc[a][b] = 0.0;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < D; n += (int64_t)gridDim.x * blockDim.x) {
    double y[Q];
#pragma unroll
    for (int b = 0; b < Q; ++b) y[b] = Y[(int64_t)b * D + n];
#pragma unroll
    for (int a = 0; a < kGramTile; ++a) {
      if (a >= na) break;
      const double x = X[(int64_t)(a0 + a) * D + n];
#pragma unroll
      for (int b = 0; b < Q; ++b) acc[a][b] = fma(x, y[b], acc[a][b]);
    }
  }
  // fixed-order block reduction, one value at a time
  __shared__ double ws[kGramThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int a = 0; a < kGramTile; ++a)
    for (int b = 0; b < Q; ++b) {
      double v = acc[a][b];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) ws[wid] = v;
      __syncthreads();
      if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kGramThreads / 32; ++w) s += ws[w];
        part[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * (kGramTile * kMaxBlock) + a * kMaxBlock + b] = s;
      }
      __syncthreads();
    }
}

// G[a * q + b] = sum over the CTAs' partials (fixed order), one thread per (a, b)
__global__ void k_gram_sum(const double *__restrict__ part, int nx, int q, int nblk, double *__restrict__ G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx * q) return;
  const int a = i / q, b = i - a * q, t = a / kGramTile;
  double s = 0.0;
  for (int c = 0; c < nblk; ++c) s += part[((int64_t)t * nblk + c) * (kGramTile * kMaxBlock) + (a % kGramTile) * kMaxBlock + b];
  G[i] = s;
}

// W_b[n] -= sum_a X_a[n] C[a * q + b]  (C: nx x q, row-major, in shared memory)
__global__ void k_sub_combo(int64_t D, const double *__restrict__ X, int nx, const double *__restrict__ C, int q,
                            double *__restrict__ W) {
  extern __shared__ double cs[];
  for (int i = threadIdx.x; i < nx * q; i += blockDim.x) cs[i] = C[i];
  __syncthreads();
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < D; n += (int64_t)gridDim.x * blockDim.x) {
    double acc[kMaxBlock];
#pragma unroll
    for (int b = 0; b < kMaxBlock; ++b) acc[b] = 0.0;
    for (int a = 0; a < nx; ++a) {
      const double x = X[(int64_t)a * D + n];
#pragma unroll
      for (int b = 0; b < kMaxBlock; ++b)
        if (b < q) acc[b] = fma(x, cs[a * q + b], acc[b]);
    }
#pragma unroll
    for (int b = 0; b < kMaxBlock; ++b)
      if (b < q) W[(int64_t)b * D + n] -= acc[b];
  }
}

// Y_b[n] = sum_{a <= b} W_a[n] R[a * q + b]  (R upper triangular: W R is the orthonormal factor)
__global__ void k_right_tri(int64_t D, const double *__restrict__ W, const double *__restrict__ R, int q,
                            double *__restrict__ Y) {
  __shared__ double rs[kMaxBlock * kMaxBlock];
  for (int i = threadIdx.x; i < q * q; i += blockDim.x) rs[i] = R[i];
  __syncthreads();
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < D; n += (int64_t)gridDim.x * blockDim.x) {
    double w[kMaxBlock];
#pragma unroll
    for (int a = 0; a < kMaxBlock; ++a) w[a] = a < q ? W[(int64_t)a * D + n] : 0.0;
#pragma unroll
    for (int b = 0; b < kMaxBlock; ++b) {
      if (b >= q) break;
      double s = 0.0;
#pragma unroll
      for (int a = 0; a <= b; ++a) s = fma(w[a], rs[a * q + b], s);
      Y[(int64_t)b * D + n] = s;
    }
  }
}

// Seeded start block for X0 == NULL: vector c is SplitMix64 uniform [-1, 1) with counter
// offset c * D (seed 0), so c = 0 equals hub_lanczos_ground's default start vector.
__global__ void k_block_start(int64_t D, int k, double *__restrict__ out) {
  const int64_t total = D * k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    out[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

struct BlockWork {
  hub_ctx *h;
  int64_t D;
  int k;
  cudaStream_t s;
  double *part = nullptr, *small = nullptr;   // Gram partials; small device matrices
  std::vector<double> hbuf;
  int gx = 1;                                 // CTAs per X-tile in k_gram_part
};

// G (nx x q, host) = X^T Y
int gram(BlockWork &w, const double *X, int nx, const double *Y, int q, std::vector<double> &G) {
  const int tiles = (nx + kGramTile - 1) / kGramTile;
  count_launch(w.h, 2);
  const dim3 g(w.gx, tiles);
  switch (q) {
    case 1: k_gram_part<1><<<g, kGramThreads, 0, w.s>>>(w.D, X, nx, Y, w.part); break;
    case 2: k_gram_part<2><<<g, kGramThreads, 0, w.s>>>(w.D, X, nx, Y, w.part); break;
    case 3: k_gram_part<3><<<g, kGramThreads, 0, w.s>>>(w.D, X, nx, Y, w.part); break;
    case 4: k_gram_part<4><<<g, kGramThreads, 0, w.s>>>(w.D, X, nx, Y, w.part); break;
    case 5: k_gram_part<5><<<g, kGramThreads, 0, w.s>>>(w.D, X, nx, Y, w.part); break;
    case 6: k_gram_part<6><<<g, kGramThreads, 0, w.s>>>(w.D, X, nx, Y, w.part); break;
    case 7: k_gram_part<7><<<g, kGramThreads, 0, w.s>>>(w.D, X, nx, Y, w.part); break;
    default: k_gram_part<8><<<g, kGramThreads, 0, w.s>>>(w.D, X, nx, Y, w.part); break;
  }
  k_gram_sum<<<(nx * q + 127) / 128, 128, 0, w.s>>>(w.part, nx, q, w.gx, w.small);
  HUB_LAUNCH_CHECK();
  G.resize((size_t)nx * q);
  HUB_CUDA(cudaMemcpyAsync(G.data(), w.small, sizeof(double) * nx * q, cudaMemcpyDeviceToHost, w.s));
  HUB_CUDA(cudaStreamSynchronize(w.s));
  return HUB_OK;
}

// W -= X C  (C: nx x q, host)
int sub_combo(BlockWork &w, const double *X, int nx, const std::vector<double> &C, double *W, int q) {
  HUB_CUDA(cudaMemcpyAsync(w.small, C.data(), sizeof(double) * nx * q, cudaMemcpyHostToDevice, w.s));
  count_launch(w.h);
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((w.D + 255) / 256, (int64_t)num_sms() * 8));
  k_sub_combo<<<g, 256, sizeof(double) * nx * q, w.s>>>(w.D, X, nx, w.small, q, W);
  HUB_LAUNCH_CHECK();
  return HUB_OK;
}

// Cholesky of the q x q Gram matrix G = R^T R (R upper); false if not positive definite to
// working precision (the block has lost rank).
bool cholesky_upper(const std::vector<double> &G, int q, std::vector<double> &R) {
  R.assign((size_t)q * q, 0.0);
  double scale = 0.0;
  for (int i = 0; i < q; ++i) scale = std::max(scale, G[i * q + i]);
  for (int j = 0; j < q; ++j) {
    double d = G[j * q + j];
    for (int p = 0; p < j; ++p) d -= R[p * q + j] * R[p * q + j];
    if (!(d > 1e-24 * std::max(scale, 1e-300))) return false;
    const double r = std::sqrt(d);
    R[j * q + j] = r;
    for (int i = j + 1; i < q; ++i) {
      double v = 0.5 * (G[j * q + i] + G[i * q + j]);
      for (int p = 0; p < j; ++p) v -= R[p * q + j] * R[p * q + i];
      R[j * q + i] = v / r;
    }
  }
  return true;
}

// inverse of an upper-triangular q x q matrix
std::vector<double> upper_inverse(const std::vector<double> &R, int q) {
  std::vector<double> X((size_t)q * q, 0.0);
  for (int j = 0; j < q; ++j) {
    X[j * q + j] = 1.0 / R[j * q + j];
    for (int i = j - 1; i >= 0; --i) {
      double s = 0.0;
      for (int p = i + 1; p <= j; ++p) s += R[i * q + p] * X[p * q + j];
      X[i * q + j] = -s / R[i * q + i];
    }
  }
  return X;
}

// W (q vectors) -> Q B with Q orthonormal (into Q) and B upper triangular, by Cholesky QR
// applied twice (B = B2 B1).  Returns false when the block has lost rank.
int chol_qr(BlockWork &w, double *W, double *Q, std::vector<double> &B, bool &ok) {
  const int q = w.k;
  std::vector<double> G, R1, R2;
  int rc;
  if ((rc = gram(w, W, q, W, q, G))) return rc;
  if (!(ok = cholesky_upper(G, q, R1))) return HUB_OK;
  HUB_CUDA(cudaMemcpyAsync(w.small, upper_inverse(R1, q).data(), sizeof(double) * q * q, cudaMemcpyHostToDevice, w.s));
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((w.D + 255) / 256, (int64_t)num_sms() * 8));
  count_launch(w.h);
  k_right_tri<<<g, 256, 0, w.s>>>(w.D, W, w.small, q, Q);
  HUB_LAUNCH_CHECK();
  if ((rc = gram(w, Q, q, Q, q, G))) return rc;
  if (!(ok = cholesky_upper(G, q, R2))) return HUB_OK;
  HUB_CUDA(cudaMemcpyAsync(w.small, upper_inverse(R2, q).data(), sizeof(double) * q * q, cudaMemcpyHostToDevice, w.s));
  count_launch(w.h);
  k_right_tri<<<g, 256, 0, w.s>>>(w.D, Q, w.small, q, W);   // W is scratch now: Q2 = Q R2^-1
  HUB_LAUNCH_CHECK();
  HUB_CUDA(cudaMemcpyAsync(Q, W, sizeof(double) * w.D * q, cudaMemcpyDeviceToDevice, w.s));
  B.assign((size_t)q * q, 0.0);                               // B = R2 R1
  for (int i = 0; i < q; ++i)
    for (int j = i; j < q; ++j) {
      double v = 0.0;
      for (int p = i; p <= j; ++p) v += R2[i * q + p] * R1[p * q + j];
      B[i * q + j] = v;
    }
  return HUB_OK;
}

// Eigen-decomposition of a symmetric n x n matrix (row-major) by cyclic Jacobi rotations:
// eigenvalues ascending into ev, eigenvectors as columns of V (row-major n x n).
void jacobi_eigen(std::vector<double> A, int n, std::vector<double> &ev, std::vector<double> &V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double a2 = A[(size_t)i * n + j] * A[(size_t)i * n + j];
        tot += a2;
        if (i != j) off += a2;
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        const double theta = 0.5 * (aqq - app) / apq;
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int r = 0; r < n; ++r) {                 // A <- A J (columns p, q)
          const double arp = A[(size_t)r * n + p], arq = A[(size_t)r * n + q];
          A[(size_t)r * n + p] = c * arp - s * arq;
          A[(size_t)r * n + q] = s * arp + c * arq;
        }
        for (int r = 0; r < n; ++r) {                 // A <- J^T A (rows p, q)
          const double apr = A[(size_t)p * n + r], aqr = A[(size_t)q * n + r];
          A[(size_t)p * n + r] = c * apr - s * aqr;
          A[(size_t)q * n + r] = s * apr + c * aqr;
        }
        for (int r = 0; r < n; ++r) {                 // V <- V J
          const double vrp = V[(size_t)r * n + p], vrq = V[(size_t)r * n + q];
          V[(size_t)r * n + p] = c * vrp - s * vrq;
          V[(size_t)r * n + q] = s * vrp + c * vrq;
        }
      }
  }
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return A[(size_t)a * n + a] < A[(size_t)b * n + b]; });
  ev.resize(n);
  std::vector<double> W((size_t)n * n);
  for (int j = 0; j < n; ++j) {
    ev[j] = A[(size_t)idx[j] * n + idx[j]];
    for (int r = 0; r < n; ++r) W[(size_t)r * n + j] = V[(size_t)r * n + idx[j]];
  }
  V.swap(W);
}

}  // namespace
}  // namespace hub

using namespace hub;

extern "C" int hub_lanczos_block(hub_t h, int k, const double *X0_dev, int steps, int n_eig, double *eig_host,
                                 double *resid_host, int *n_found, void *stream) {
  int rc = ready(h, "hub_lanczos_block");
  if (rc) return rc;
  if (k < 1 || k > kMaxBlock || steps < 1 || (int64_t)k * steps > kMaxKrylov || n_eig < 1 || !eig_host || !n_found)
    return fail(HUB_ERR_ARG, "hub_lanczos_block: need 1 <= k <= 8, steps >= 1, k * steps <= 512, n_eig >= 1, "
                             "eig_host and n_found");
  const int64_t D = vec_len(h);
  if (D < (int64_t)k) return fail(HUB_ERR_ARG, "hub_lanczos_block: block larger than the space");
  cudaStream_t s = (cudaStream_t)stream;
  BlockWork w;
  w.h = h;
  w.D = D;
  w.k = k;
  w.s = s;
  w.gx = (int)std::max<int64_t>(1, std::min<int64_t>((D + kGramThreads - 1) / kGramThreads, (int64_t)num_sms() * 2));
  // device memory: steps + 1 blocks of Q, one scratch block, Gram partials, small matrices
  const int64_t nvec = (int64_t)(steps + 2) * k;
  double *Qall = nullptr, *part = nullptr, *small = nullptr;
  const int tiles = (int)((steps + 1) * k + kGramTile - 1) / kGramTile;
  if (!dev_alloc((void **)&Qall, sizeof(double) * D * nvec, "block Lanczos vectors")) return HUB_ERR_OOM;
  if (!dev_alloc((void **)&part, sizeof(double) * (size_t)tiles * w.gx * kGramTile * kMaxBlock, "Gram partials") ||
      !dev_alloc((void **)&small, sizeof(double) * (size_t)(steps + 1) * k * k, "block coefficients")) {
    dev_free(Qall);
    dev_free(part);
    return HUB_ERR_OOM;
  }
  w.part = part;
  w.small = small;
  auto Q = [&](int j) { return Qall + (int64_t)j * k * D; };   // block j (j = 0 .. steps)
  double *W = Q(steps + 1);
  std::vector<std::vector<double>> A, B;                         // diagonal and sub-diagonal blocks
  auto body = [&]() -> int {
    int rc2;
    if (X0_dev) {
      HUB_CUDA(cudaMemcpyAsync(W, X0_dev, sizeof(double) * D * k, cudaMemcpyDeviceToDevice, s));
    } else {
      count_launch(h);
      k_block_start<<<num_sms() * 8, 256, 0, s>>>(D, k, W);
      HUB_LAUNCH_CHECK();
    }
    if (h->k0)
      for (int c = 0; c < k; ++c)
        if ((rc2 = k0_project_inplace(h, W + (int64_t)c * D, s))) return rc2;
    std::vector<double> Bj;
    bool ok = true;
    if ((rc2 = chol_qr(w, W, Q(0), Bj, ok))) return rc2;
    if (!ok) return fail(HUB_ERR_ARG, "hub_lanczos_block: the start vectors are linearly dependent");
    for (int j = 0; j < steps; ++j) {
      for (int c = 0; c < k; ++c)
        if ((rc2 = apply_launch(h, Q(j) + (int64_t)c * D, W + (int64_t)c * D, s))) return rc2;
      if (j > 0) {                                   // W -= Q_{j-1} B_{j-1}^T
        std::vector<double> Bt((size_t)k * k);
        for (int a = 0; a < k; ++a)
          for (int b = 0; b < k; ++b) Bt[a * k + b] = B[j - 1][b * k + a];
        if ((rc2 = sub_combo(w, Q(j - 1), k, Bt, W, k))) return rc2;
      }
      std::vector<double> Aj;
      if ((rc2 = gram(w, Q(j), k, W, k, Aj))) return rc2;
      for (int a = 0; a < k; ++a)                    // symmetrise (exact arithmetic gives A_j = A_j^T)
        for (int b = a + 1; b < k; ++b) Aj[a * k + b] = Aj[b * k + a] = 0.5 * (Aj[a * k + b] + Aj[b * k + a]);
      if ((rc2 = sub_combo(w, Q(j), k, Aj, W, k))) return rc2;
      A.push_back(Aj);
      for (int pass = 0; pass < 2; ++pass) {         // full re-orthogonalisation against Q_0 .. Q_j
        std::vector<double> C;
        if ((rc2 = gram(w, Q(0), (j + 1) * k, W, k, C))) return rc2;
        if ((rc2 = sub_combo(w, Q(0), (j + 1) * k, C, W, k))) return rc2;
      }
      if ((rc2 = chol_qr(w, W, Q(j + 1), Bj, ok))) return rc2;
      if (!ok) break;                                // invariant subspace: T is complete
      B.push_back(Bj);
    }
    return HUB_OK;
  };
  rc = body();
  const cudaError_t se = cudaStreamSynchronize(s);
  dev_free(Qall);
  dev_free(part);
  dev_free(small);
  if (rc) return rc;
  if (se != cudaSuccess) return cuda_fail(se, "hub_lanczos_block", __FILE__, __LINE__);

  // T: block tridiagonal, n = k * (number of diagonal blocks)
  const int nb = (int)A.size(), n = nb * k;
  std::vector<double> T((size_t)n * n, 0.0);
  for (int j = 0; j < nb; ++j)
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) {
        T[(size_t)(j * k + a) * n + j * k + b] = A[j][a * k + b];
        if (j + 1 < nb) {                            // H Q_j has Q_{j+1} B_j: T[(j+1)k + a, jk + b] = B_j[a][b]
          T[(size_t)((j + 1) * k + a) * n + j * k + b] = B[j][a * k + b];
          T[(size_t)(j * k + b) * n + (j + 1) * k + a] = B[j][a * k + b];
        }
      }
  std::vector<double> ev, V;
  jacobi_eigen(T, n, ev, V);
  const int m = std::min(n_eig, n);
  for (int i = 0; i < m; ++i) {
    eig_host[i] = ev[i];
    if (resid_host) {
      // |H y - theta y| = |B_last s_last| (zero when the space became invariant)
      double r2 = 0.0;
      if ((int)B.size() == nb) {
        for (int a = 0; a < k; ++a) {
          double v = 0.0;
          for (int b = 0; b < k; ++b) v += B[nb - 1][a * k + b] * V[(size_t)((nb - 1) * k + b) * n + i];
          r2 += v * v;
        }
      }
      resid_host[i] = std::sqrt(r2);
    }
  }
  *n_found = m;
  return HUB_OK;
}
