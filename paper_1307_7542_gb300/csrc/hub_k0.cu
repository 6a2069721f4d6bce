// hub_k0.cu -- the k = 0 sector of a translation-invariant chain (Sec. V).
//
// T moves every electron one site down the chain, T c+_i T^-1 = c+_{i-1} (site 0 to site
// M-1), the direction of Tables I and II.  On a spin string x with N electrons (sites in
// ascending order) one step is the rotation x -> (x >> 1) | (x & 1) << (M-1) with sign
// (-1)^(N-1) when site 0 was occupied; after t steps the sign is (-1)^((N-1) c) with c the
// electrons of x on sites 0 .. t-1.
//
// Layout ("row form").  The up strings fall into translation cycles; the smallest member of
// a cycle is its representative R_i (Sec. V), i = 0 .. rows-1 in ascending order, with
// period P_i.  A k = 0 vector Psi of the full two-spin space is determined by its values on
// the pairs (R_i, d), d any down string, and is stored as
//     X[i * cols + r] = sqrt(P_i) * Psi(R_i, d_r),   cols = count_dn, r the rank of d_r,
// so that the Euclidean inner product of two such arrays equals that of the two-spin
// vectors.  When P_i = M every pair (R_i, d) lies in a different cycle of T and row i is
// free.  When P_i < M, T^P_i maps row i to itself (T^P_i |R_i> = b_i |R_i>), and the
// entries of one T^P_i-cycle of the row are tied together; a cycle whose closing sign is -1
// has no k = 0 state and is zero.  The library keeps those few rows consistent: every
// product and every start vector is projected onto them, with each cycle's average summed
// in one fixed order so that the tied entries agree bit for bit.
//
// The k = pi sector (T Psi = -Psi, M even) uses the same layout: every relation
// Psi(T^t c) = tau Psi(c) of the k = 0 sector gains the factor (-1)^t, so the up-hop
// coefficients take (-1)^t and the closing sign of a short row b_i becomes (-1)^P_i b_i.
//
// Product in row form (Sec. V with Eq. 11): for (i, d)
//     Y = (U popc(R_i & d) + eps (N_up + N_dn)) X[i, d]                diagonal
//       + sum_d' H_dn[d, d'] X[i, d']                                    down hops, in-row
//       + sum_{u'} H_up[R_i, u'] s sqrt(P_i / P_i') s_e X[i', e]          up hops
// where T^t |R_i'> = s |u'> (R_i' the representative of u', t < P_i') and e = T^-t d with
// T^t |e> = s_e |d>.  The up-hop list of each row (i', t, coefficient) is built on the host;
// the (rank of T^-t d, s_e) table for all t < M and all down strings on the device.
#include <algorithm>
#include <cmath>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "hub_internal.cuh"

namespace hub {

int ready(const hub_ctx *h, const char *who);

constexpr int kK0Threads = 256;

struct K0State {
  int64_t rows = 0, cols = 0, dim = 0;
  std::vector<uint32_t> rep_h;
  std::vector<int32_t> per_h;
  uint32_t *rep = nullptr;      // [rows] up representatives, ascending
  int32_t *per = nullptr;       // [rows] their periods
  int32_t *eb = nullptr;        // [rows] sign of T^P_i on R_i, times omega^P_i
  int omega = 1;                // e^{ik}: 1 for k = 0, -1 for k = pi
  int32_t *uh_ptr = nullptr;    // [rows + 1] up-hop list of each row
  int32_t *uh_row = nullptr;    // [n_uh] target row i'
  int32_t *uh_t = nullptr;      // [n_uh] translation t
  double *uh_val = nullptr;     // [n_uh] H_up[R_i, u'] s sqrt(P_i / P_i')
  uint32_t *rot = nullptr;      // [M * cols] rank of T^-t d | (s_e = -1) << 31
  int32_t *short_rows = nullptr;   // rows with P_i < M
  int n_short = 0;
  double *scratch = nullptr;    // [n_short * cols]
  unsigned long long *d_count = nullptr;
  double diag0 = 0.0;           // eps (N_up + N_dn) for uniform eps
};

struct K0View {
  int M;
  int64_t rows, cols;
  const uint32_t *rep;
  const int32_t *per, *eb;
  const int32_t *uh_ptr, *uh_row, *uh_t;
  const double *uh_val;
  const uint32_t *rot;
  const int32_t *rp_dn, *col_dn;
  const double *val_dn;
  const uint32_t *basis_dn;
  double U0, diag0;
};

static K0View k0_view(const hub_ctx *h) {
  const K0State *k = h->k0;
  const Ham H = h->view();
  K0View v{};
  v.M = h->M;
  v.rows = k->rows;
  v.cols = k->cols;
  v.rep = k->rep;
  v.per = k->per;
  v.eb = k->eb;
  v.uh_ptr = k->uh_ptr;
  v.uh_row = k->uh_row;
  v.uh_t = k->uh_t;
  v.uh_val = k->uh_val;
  v.rot = k->rot;
  v.rp_dn = H.rp_dn;
  v.col_dn = H.col_dn;
  v.val_dn = H.val_dn;
  v.basis_dn = H.basis_dn;
  v.U0 = h->U0;
  v.diag0 = k->diag0;
  return v;
}

// ---------------------------------------------------------------------------------------
// Device side
// ---------------------------------------------------------------------------------------

// (rank of e = T^-t d, s_e) for every t < M and every down string d of rank r.
__global__ void k_k0_rot(int M, int N, int64_t cols, const uint32_t *__restrict__ basis,
                         const uint64_t *__restrict__ C, uint32_t *__restrict__ rot) {
  const uint32_t mask = (uint32_t)((1ull << M) - 1);
  const int64_t n = (int64_t)M * cols;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(k / cols);
    const uint32_t d = basis[k - (int64_t)t * cols];
    const uint32_t e = t ? (((d << t) | (d >> (M - t))) & mask) : d;
    const int c = __popc(e & (uint32_t)((1ull << t) - 1));
    const bool neg = ((N - 1) & 1) && (c & 1);
    rot[k] = rank_of(e, C) | (neg ? 0x80000000u : 0u);
  }
}

// Member g of the T^P-cycle of column r in a row with period P and closing sign b:
// position of T^-(gP) d and the sign beta with Psi(R, d) = beta Psi(R, T^-(gP) d).
__device__ __forceinline__ uint32_t k0_member(const K0View &K, int P, int b, int g, int64_t r, int *sign) {
  const uint32_t w = __ldg(K.rot + (int64_t)(g * P) * K.cols + r);
  int s = (w >> 31) ? -1 : 1;
  if (b < 0 && (g & 1)) s = -s;
  *sign = s;
  return w & 0x7fffffffu;
}

// Row value of the product at (i, r) before the projection of short rows.
__device__ __forceinline__ double k0_row_value(const K0View &K, int64_t i, int64_t r, const double *__restrict__ x) {
  const double *xi = x + i * K.cols;
  double acc = fma(K.U0, (double)__popc(__ldg(K.rep + i) & __ldg(K.basis_dn + r)), K.diag0) * xi[r];
  const int k0 = __ldg(K.rp_dn + r), k1 = __ldg(K.rp_dn + r + 1);
  for (int k = k0; k < k1; ++k) acc = fma(__ldg(K.val_dn + k), xi[__ldg(K.col_dn + k)], acc);
  const int h0 = __ldg(K.uh_ptr + i), h1 = __ldg(K.uh_ptr + i + 1);
  for (int k = h0; k < h1; ++k) {
    const uint32_t w = __ldg(K.rot + (int64_t)__ldg(K.uh_t + k) * K.cols + r);
    const double c = __ldg(K.uh_val + k);
    acc = fma((w >> 31) ? -c : c, x[(int64_t)__ldg(K.uh_row + k) * K.cols + (w & 0x7fffffffu)], acc);
  }
  return acc;
}

// Projection of a short row onto its tied cycles at column r: the cycle's average, summed
// from its smallest-rank member in the order g = 0, 1, ..., times the sign relating r to
// that member; 0 for a cycle that closes with sign -1.  value(pos) gives the unprojected
// entry of the row at column pos.
template <class F>
__device__ __forceinline__ double k0_projected(const K0View &K, int64_t i, int64_t r, F value) {
  const int P = __ldg(K.per + i), b = __ldg(K.eb + i), G = K.M / P;
  int64_t c = r;
  int cs = 1;
  for (int g = 1; g < G; ++g) {
    int s;
    const int64_t pos = k0_member(K, P, b, g, r, &s);
    if (pos == r && s < 0) return 0.0;
    if (pos < c) {
      c = pos;
      cs = s;
    }
  }
  double sum = value(c);
  for (int g = 1; g < G; ++g) {
    int s;
    const int64_t pos = k0_member(K, P, b, g, c, &s);
    const double v = value(pos);
    sum += s < 0 ? -v : v;
  }
  const double avg = sum / (double)G;
  return cs < 0 ? -avg : avg;
}

__global__ void __launch_bounds__(kK0Threads) k_k0_apply(K0View K, const double *__restrict__ x,
                                                         double *__restrict__ y) {
  const int64_t chunks = (K.cols + kK0Threads - 1) / kK0Threads;
  const int64_t tiles = K.rows * chunks;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t i = tile / chunks;
    const int64_t r = (tile - i * chunks) * kK0Threads + threadIdx.x;
    if (r >= K.cols) continue;
    double v;
    if (__ldg(K.per + i) == K.M)
      v = k0_row_value(K, i, r, x);
    else
      v = k0_projected(K, i, r, [&](int64_t pos) { return k0_row_value(K, i, pos, x); });
    y[i * K.cols + r] = v;
  }
}

// scratch[s, r] = x[short_rows[s], r]
__global__ void k_k0_gather_short(int64_t cols, int n_short, const int32_t *__restrict__ short_rows,
                                  const double *__restrict__ x, double *__restrict__ scratch) {
  const int64_t n = (int64_t)n_short * cols;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = k / cols;
    scratch[k] = x[(int64_t)short_rows[s] * cols + (k - s * cols)];
  }
}

// y[short_rows[s], r] = projection of scratch row s at r
__global__ void k_k0_project_short(K0View K, int n_short, const int32_t *__restrict__ short_rows,
                                   const double *__restrict__ scratch, double *__restrict__ y) {
  const int64_t n = (int64_t)n_short * K.cols;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = k / K.cols, r = k - s * K.cols;
    const double *src = scratch + s * K.cols;
    const int64_t i = short_rows[s];
    y[i * K.cols + r] = k0_projected(K, i, r, [&](int64_t pos) { return src[pos]; });
  }
}

// Number of k = 0 states in the short rows: columns that are the smallest member of a
// cycle that does not close with sign -1.
__global__ void k_k0_count_short(K0View K, int n_short, const int32_t *__restrict__ short_rows,
                                 unsigned long long *__restrict__ count) {
  const int64_t n = (int64_t)n_short * K.cols;
  unsigned long long mine = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = k / K.cols, r = k - s * K.cols;
    const int64_t i = short_rows[s];
    const int P = K.per[i], b = K.eb[i], G = K.M / P;
    bool least = true, null = false;
    for (int g = 1; g < G; ++g) {
      int sg;
      const int64_t pos = k0_member(K, P, b, g, r, &sg);
      if (pos < r) least = false;
      if (pos == r && sg < 0) null = true;
    }
    if (least && !null) ++mine;
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(count, mine);
}

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------

static inline uint32_t step_T(uint32_t x, int M) { return (x >> 1) | ((x & 1u) << (M - 1)); }
static inline int step_sign(uint32_t x, int N) { return ((x & 1u) && ((N - 1) & 1)) ? -1 : 1; }

void k0_release(hub_ctx *h) {
  K0State *k = h->k0;
  if (!k) return;
  dev_free(k->rep);
  dev_free(k->per);
  dev_free(k->eb);
  dev_free(k->uh_ptr);
  dev_free(k->uh_row);
  dev_free(k->uh_t);
  dev_free(k->uh_val);
  dev_free(k->rot);
  dev_free(k->short_rows);
  dev_free(k->scratch);
  dev_free(k->d_count);
  delete k;
  h->k0 = nullptr;
}

// Drop the vectors sized for the previous sector layout.
static void release_vectors(hub_ctx *h) {
  for (int k = 0; k < 3; ++k) {
    dev_free(h->work[k]);
    h->work[k] = nullptr;
  }
  dev_free(h->hx);
  dev_free(h->hy);
  h->hx = h->hy = nullptr;
}

void k0_leave(hub_ctx *h) {
  if (!h->k0) return;
  k0_release(h);
  release_vectors(h);
}

int64_t vec_len(const hub_ctx *h) {
  if (h->k0) return h->k0->rows * h->k0->cols;
  return h->count[0] * h->count[1];
}

// H must commute with T: every bond moved one site down is a bond with the same t, and U and
// eps are the same on every site.
static int check_invariant(const hub_ctx *h) {
  const int M = h->M;
  std::map<std::pair<int, int>, double> bonds;
  for (int b = 0; b < h->n_bonds; ++b) {
    const int i = h->bonds[2 * b], j = h->bonds[2 * b + 1];
    bonds[{std::min(i, j), std::max(i, j)}] = h->t[b];
  }
  for (int b = 0; b < h->n_bonds; ++b) {
    const int i = (h->bonds[2 * b] + M - 1) % M, j = (h->bonds[2 * b + 1] + M - 1) % M;
    const auto it = bonds.find({std::min(i, j), std::max(i, j)});
    if (it == bonds.end() || it->second != h->t[b])
      return fail(HUB_ERR_ARG, "hub_set_symmetry: the bonds are not invariant under the translation i -> i-1 mod M");
  }
  if (!h->uniform_U) return fail(HUB_ERR_ARG, "hub_set_symmetry: U differs between sites");
  for (int i = 1; i < M; ++i)
    if (h->eps[i] != h->eps[0]) return fail(HUB_ERR_ARG, "hub_set_symmetry: eps differs between sites");
  return HUB_OK;
}

static int k0_build(hub_ctx *h, int omega) {
  const int M = h->M, Nu = h->N[0], Nd = h->N[1];
  K0State *k = new (std::nothrow) K0State();
  if (!k) return fail(HUB_ERR_OOM, "hub_set_symmetry: host allocation failed");
  h->k0 = k;
  k->omega = omega;
  k->cols = h->count[1];
  k->diag0 = (h->eps.empty() ? 0.0 : h->eps[0]) * (double)(Nu + Nd);

  // up representatives (smallest member of each cycle), ascending, with periods and signs
  std::vector<uint32_t> reps;
  std::vector<int32_t> per, eb;
  {
    const uint64_t limit = 1ull << M;
    uint64_t u = Nu == 0 ? 0 : (1ull << Nu) - 1;
    while (u < limit) {
      const uint32_t x = (uint32_t)u;
      uint32_t c = x, least = x;
      int P = M;
      for (int s = 1; s <= M; ++s) {
        c = step_T(c, M);
        if (c == x) {
          P = s;
          break;
        }
        least = std::min(least, c);
      }
      if (least == x) {
        int sg = 1;
        uint32_t y = x;
        for (int s = 0; s < P; ++s) {
          sg *= step_sign(y, Nu);
          y = step_T(y, M);
        }
        reps.push_back(x);
        per.push_back(P);
        eb.push_back((omega < 0 && (P & 1)) ? -sg : sg);
      }
      if (Nu == 0) break;
      const uint64_t lo = u & (~u + 1), r = u + lo;   // next string with Nu bits (Gosper)
      u = (((r ^ u) >> 2) / lo) | r;
    }
  }
  k->rows = (int64_t)reps.size();
  k->rep_h = reps;
  k->per_h = per;

  // size check before any large allocation
  size_t free_b = 0, total_b = 0;
  HUB_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const double row_form_bytes = 8.0 * (double)k->rows * (double)k->cols;
  if (row_form_bytes > (double)free_b) return fail(HUB_ERR_OOM, "hub_set_symmetry: one k = 0 vector does not fit");

  // up-hop lists
  std::vector<int32_t> uh_ptr(1, 0), uh_row, uh_t;
  std::vector<double> uh_val;
  for (size_t i = 0; i < reps.size(); ++i) {
    const uint32_t R = reps[i];
    for (int b = 0; b < h->n_bonds; ++b) {
      const int a = h->bonds[2 * b], c = h->bonds[2 * b + 1];
      if (((R >> a) & 1u) == ((R >> c) & 1u)) continue;
      const uint32_t u2 = R ^ ((1u << a) | (1u << c));
      const int lo = std::min(a, c), hi = std::max(a, c);
      const uint32_t between = ((1u << hi) - 1u) & ~((2u << lo) - 1u);
      const double val = -h->t[b] * ((popc32(R & between) & 1) ? -1.0 : 1.0);
      uint32_t least = u2, cur = u2;
      for (int s = 1; s < M; ++s) {
        cur = step_T(cur, M);
        least = std::min(least, cur);
      }
      const auto it = std::lower_bound(reps.begin(), reps.end(), least);
      if (it == reps.end() || *it != least) return fail(HUB_ERR_CUDA, "hub_set_symmetry: representative not found");
      const int i2 = (int)(it - reps.begin());
      int t = 0, sg = 1;
      cur = least;
      while (cur != u2 && t < per[i2]) {
        sg *= step_sign(cur, Nu);
        cur = step_T(cur, M);
        ++t;
      }
      if (cur != u2) return fail(HUB_ERR_CUDA, "hub_set_symmetry: translation not found");
      uh_row.push_back(i2);
      uh_t.push_back(t);
      if (omega < 0 && (t & 1)) sg = -sg;
      uh_val.push_back(val * sg * std::sqrt((double)per[i] / (double)per[i2]));
    }
    uh_ptr.push_back((int32_t)uh_row.size());
  }
  std::vector<int32_t> shorts;
  for (size_t i = 0; i < reps.size(); ++i)
    if (per[i] < M) shorts.push_back((int32_t)i);
  k->n_short = (int)shorts.size();

  const size_t n_uh = std::max<size_t>(uh_row.size(), 1);
  const int64_t nrot = (int64_t)M * k->cols;
  if (!dev_alloc((void **)&k->rep, sizeof(uint32_t) * std::max<int64_t>(k->rows, 1), "k = 0 representatives") ||
      !dev_alloc((void **)&k->per, sizeof(int32_t) * std::max<int64_t>(k->rows, 1), "k = 0 periods") ||
      !dev_alloc((void **)&k->eb, sizeof(int32_t) * std::max<int64_t>(k->rows, 1), "k = 0 signs") ||
      !dev_alloc((void **)&k->uh_ptr, sizeof(int32_t) * (k->rows + 1), "k = 0 up hops") ||
      !dev_alloc((void **)&k->uh_row, sizeof(int32_t) * n_uh, "k = 0 up hops") ||
      !dev_alloc((void **)&k->uh_t, sizeof(int32_t) * n_uh, "k = 0 up hops") ||
      !dev_alloc((void **)&k->uh_val, sizeof(double) * n_uh, "k = 0 up hops") ||
      !dev_alloc((void **)&k->rot, sizeof(uint32_t) * std::max<int64_t>(nrot, 1), "k = 0 translation table") ||
      !dev_alloc((void **)&k->short_rows, sizeof(int32_t) * std::max<size_t>(shorts.size(), 1), "k = 0 short rows") ||
      !dev_alloc((void **)&k->scratch, sizeof(double) * std::max<int64_t>(k->n_short * k->cols, 1), "k = 0 scratch") ||
      !dev_alloc((void **)&k->d_count, sizeof(unsigned long long), "k = 0 counter"))
    return HUB_ERR_OOM;
  if (k->rows) {
    HUB_CUDA(cudaMemcpy(k->rep, reps.data(), sizeof(uint32_t) * k->rows, cudaMemcpyHostToDevice));
    HUB_CUDA(cudaMemcpy(k->per, per.data(), sizeof(int32_t) * k->rows, cudaMemcpyHostToDevice));
    HUB_CUDA(cudaMemcpy(k->eb, eb.data(), sizeof(int32_t) * k->rows, cudaMemcpyHostToDevice));
  }
  HUB_CUDA(cudaMemcpy(k->uh_ptr, uh_ptr.data(), sizeof(int32_t) * (k->rows + 1), cudaMemcpyHostToDevice));
  if (!uh_row.empty()) {
    HUB_CUDA(cudaMemcpy(k->uh_row, uh_row.data(), sizeof(int32_t) * uh_row.size(), cudaMemcpyHostToDevice));
    HUB_CUDA(cudaMemcpy(k->uh_t, uh_t.data(), sizeof(int32_t) * uh_t.size(), cudaMemcpyHostToDevice));
    HUB_CUDA(cudaMemcpy(k->uh_val, uh_val.data(), sizeof(double) * uh_val.size(), cudaMemcpyHostToDevice));
  }
  if (!shorts.empty())
    HUB_CUDA(cudaMemcpy(k->short_rows, shorts.data(), sizeof(int32_t) * shorts.size(), cudaMemcpyHostToDevice));
  const int sms = num_sms();
  if (nrot > 0) {
    k_k0_rot<<<(int)std::min<int64_t>((nrot + 255) / 256, (int64_t)sms * 32), 256>>>(M, Nd, k->cols, h->basis[1],
                                                                                   h->binom, k->rot);
    HUB_LAUNCH_CHECK();
  }
  // dimension: free rows count fully, short rows by their cycles
  k->dim = (k->rows - k->n_short) * k->cols;
  if (k->n_short && k->cols) {
    HUB_CUDA(cudaMemset(k->d_count, 0, sizeof(unsigned long long)));
    const int64_t n = (int64_t)k->n_short * k->cols;
    k_k0_count_short<<<(int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 32), 256>>>(k0_view(h), k->n_short,
                                                                                       k->short_rows, k->d_count);
    HUB_LAUNCH_CHECK();
    unsigned long long c = 0;
    HUB_CUDA(cudaMemcpy(&c, k->d_count, sizeof(c), cudaMemcpyDeviceToHost));
    k->dim += (int64_t)c;
  }
  HUB_CUDA(cudaDeviceSynchronize());
  return HUB_OK;
}

int k0_apply(hub_ctx *h, const double *x, double *y, cudaStream_t s) {
  const K0State *k = h->k0;
  if (k->rows == 0 || k->cols == 0) return HUB_OK;
  const int64_t tiles = k->rows * ((k->cols + kK0Threads - 1) / kK0Threads);
  const int grid = (int)std::min<int64_t>(tiles, (int64_t)num_sms() * 16);
  count_launch(h);
  k_k0_apply<<<grid, kK0Threads, 0, s>>>(k0_view(h), x, y);
  HUB_LAUNCH_CHECK();
  return HUB_OK;
}

int k0_project_inplace(hub_ctx *h, double *x, cudaStream_t s) {
  const K0State *k = h->k0;
  if (k->n_short == 0 || k->cols == 0) return HUB_OK;
  const int64_t n = (int64_t)k->n_short * k->cols;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 16);
  count_launch(h, 2);
  k_k0_gather_short<<<grid, 256, 0, s>>>(k->cols, k->n_short, k->short_rows, x, k->scratch);
  HUB_LAUNCH_CHECK();
  k_k0_project_short<<<grid, 256, 0, s>>>(k0_view(h), k->n_short, k->short_rows, k->scratch, x);
  HUB_LAUNCH_CHECK();
  return HUB_OK;
}

}  // namespace hub

using namespace hub;

extern "C" int hub_set_symmetry(hub_t h, int sym) {
  if (!h) return fail(HUB_ERR_ARG, "hub_set_symmetry: NULL handle");
  if (sym != HUB_SYM_NONE && sym != HUB_SYM_K0 && sym != HUB_SYM_KPI)
    return fail(HUB_ERR_ARG, "hub_set_symmetry: unknown symmetry");
  if (sym == HUB_SYM_NONE) {
    k0_leave(h);
    return HUB_OK;
  }
  int rc = ready(h, "hub_set_symmetry");
  if (rc) return rc;
  if ((rc = check_invariant(h))) return rc;
  if (sym == HUB_SYM_KPI && (h->M & 1)) return fail(HUB_ERR_ARG, "hub_set_symmetry: k = pi needs an even M");
  k0_release(h);
  release_vectors(h);
  rc = k0_build(h, sym == HUB_SYM_KPI ? -1 : 1);
  if (rc) k0_release(h);
  return rc;
}

extern "C" int hub_k_dims(hub_t h, int64_t *rows, int64_t *cols, int64_t *dim) {
  if (!h) return fail(HUB_ERR_ARG, "hub_k_dims: NULL handle");
  if (!h->k0) return fail(HUB_ERR_STATE, "hub_k_dims: no momentum sector is active (hub_set_symmetry)");
  if (rows) *rows = h->k0->rows;
  if (cols) *cols = h->k0->cols;
  if (dim) *dim = h->k0->dim;
  return HUB_OK;
}

extern "C" int hub_k_reps(hub_t h, uint32_t *rep_host, int32_t *period_host) {
  if (!h) return fail(HUB_ERR_ARG, "hub_k_reps: NULL handle");
  if (!h->k0) return fail(HUB_ERR_STATE, "hub_k_reps: no momentum sector is active (hub_set_symmetry)");
  const K0State *k = h->k0;
  for (int64_t i = 0; i < k->rows; ++i) {
    if (rep_host) rep_host[i] = k->rep_h[i];
    if (period_host) period_host[i] = k->per_h[i];
  }
  return HUB_OK;
}

extern "C" int hub_k_project(hub_t h, const double *x_dev, double *y_dev, void *stream) {
  if (!h) return fail(HUB_ERR_ARG, "hub_k_project: NULL handle");
  if (!h->k0) return fail(HUB_ERR_STATE, "hub_k_project: no momentum sector is active (hub_set_symmetry)");
  if (!x_dev || !y_dev) return fail(HUB_ERR_ARG, "hub_k_project: NULL vector");
  const int64_t D = vec_len(h);
  if (x_dev != y_dev && x_dev < y_dev + D && y_dev < x_dev + D)
    return fail(HUB_ERR_ARG, "hub_k_project: x and y overlap without being equal");
  cudaStream_t s = (cudaStream_t)stream;
  if (x_dev != y_dev && D) HUB_CUDA(cudaMemcpyAsync(y_dev, x_dev, sizeof(double) * D, cudaMemcpyDeviceToDevice, s));
  return k0_project_inplace(h, y_dev, s);
}
