// hub_k0.cu -- momentum sectors of translation-invariant lattices (Sec. V).
//
// Sec. V reduces the chain by its translation T c+_i T^-1 = c+_{i-1} (site 0 to site M-1, the
// direction of Tables I and II) to the k = 0 space.  The same construction holds for any
// abelian group G of site permutations that leaves H unchanged (the two translations of a
// torus, ...) and any real character chi of G (chi(g) = +-1; for the chain k = 0 and k = pi):
// the sector is {Psi : g Psi = chi(g) Psi for all g}.  An element g acts on a spin string x as
// g|x> = sign |x'>, x' the permuted sites and sign the parity of reordering the images of the
// occupied sites (creation operators in ascending site order).  A string's orbit has
// |G| / |S| members (S its stabiliser, on which g|x> = sigma(g)|x>); its smallest member is
// the representative.
//
// Layout ("row form", the order of Table I).  Rows: the up representatives R_i, ascending,
// orbit sizes P_i.  Columns: the down representatives R_j, ascending, each followed by the
// rest of its orbit: column c = (j, k) stands for the signed state c_k |R_j>, c_0 = 1, c_k the
// smallest element of the k-th coset of S_j.  A state of the sector is stored as
//     X[i * cols + c] = sqrt(P_i) <R_i (x) c_k R_j | Psi>,        cols = count_dn,
// and the plain dot product of two such arrays equals the inner product of the states.  When
// S_i is trivial every column of row i belongs to a different orbit and the row is free.
// Otherwise the elements h of S_i tie the entries of each column block, X[i, (j, k)] =
// chi(h) sigma_i(h) sigma' X[i, (j, k')] with h c_k = c_k' h' (h' in S_j, sigma' = sigma_j(h'));
// an orbit that meets itself with sign -1 has no state in the sector and is zero.  The
// library keeps those few rows consistent: every product and every start vector is projected
// onto them, each orbit's average summed in one fixed order so that tied entries agree bit
// for bit.  How an element moves the members of a block depends only on the block's
// stabiliser and its signs (its "type"): one small table per type, tab[e][k] = (k', sigma')
// with e c_k = c_k' h', sigma' = sigma_j(h').  For the chain a block is a cycle of period P_j
// and the table is the cyclic shift k -> k - t mod P_j.
//
// Product (Sec. V with Eq. 11): for entry (i, c), c = (j, k), d the string of c_k R_j,
//     Y = (U popc(R_i & d) + eps (N_up + N_dn)) X[i, c]                           diagonal
//       + sum_c' H_dn[d, d'] s_c s_c' X[i, c']                                      down hops
//       + sum_{u'} H_up[R_i, u'] s chi(g) sqrt(P_i / P_i') sigma' X[i', (j, k')]      up hops
// where s_c is the sign of c_k |R_j> relative to |d>, g |R_i'> = s |u'> (R_i' the
// representative of u'), and (k', sigma') = tab_j[g^-1][k].  The up-hop list of each row
// (i', g^-1, coefficient), the tables and the down hopping matrix in this column order are
// built on the host.
//
// Integer accumulation.  GB300 issues FP64 at about 1/70 of its FP32 and integer rates, and
// the product above is about 22 FP64 multiply-adds per entry.  With uniform t every hop term
// is -t times +-x, so the entry is diag x + (-t) S with S a signed sum of gathered values.
// S is formed in 64-bit fixed point on the integer pipe: the point sits at the largest
// exponent among the entry's own terms (the accumulator is shifted down whenever a larger one
// arrives), each term's 53-bit significand shifted in with s0 guard bits, s0 chosen so that
// no sum of the entry's terms can overflow.  The only rounding is the truncation of each
// aligned term, below 2^-(52+s0) of the largest term, far inside the 1e-13 (|H||x|)_n bound;
// one int64 -> FP64 conversion and two FP64 multiply-adds finish the entry.  Hops whose
// coefficient is not +-t (rows with a nontrivial stabiliser and hops into them, factor
// sqrt(P_i / P_i')) stay in FP64.  HUB_MODE_FP64 selects a kernel with FP64 multiply-adds
// throughout (also used when t is not uniform).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "hub_group.h"
#include "hub_internal.cuh"

namespace hub {

int ready(const hub_ctx *h, const char *who);

constexpr int kK0Threads = 256;
// uh_t word: element g^-1 in bits 0-7; integer path: the hop's coefficient is +-t (bit 8),
// and its sign relative to -t (bit 9)
constexpr int kHopUnit = 1 << 8, kHopNeg = 1 << 9;
// column word: k in bits 0-7, block type in bits 8-15
// table entry: k' in bits 0-7, sigma' = -1 in bit 15

struct K0State {
  int64_t rows = 0, cols = 0, dim = 0;
  int g = 0;                    // group order
  std::vector<uint32_t> rep_h, col_bits_h;
  std::vector<int32_t> per_h, col_sign_h;
  uint32_t *rep = nullptr;      // [rows] up representatives, ascending
  int32_t *per = nullptr;       // [rows] orbit sizes
  int32_t *st_ptr = nullptr;    // [rows + 1] stabiliser list of each row (identity left out)
  int32_t *st = nullptr;        // element | (chi(h) sigma_i(h) = -1) << 8
  int32_t *uh_ptr = nullptr;    // [rows + 1] up-hop list of each row
  int32_t *uh_row = nullptr;    // [n_uh] target row i'
  int32_t *uh_t = nullptr;      // [n_uh] element g^-1 and flags
  double *uh_val = nullptr;     // [n_uh] H_up[R_i, u'] s chi(g) sqrt(P_i / P_i')
  uint32_t *cinfo = nullptr;    // [cols] k | type << 8
  uint32_t *cbits = nullptr;    // [cols] down string of the column
  int32_t *tab_off = nullptr;   // [types] start of each type's table; its block size follows
  uint16_t *tab = nullptr;      // tables, [e][k] per type
  int32_t *krp = nullptr;       // [cols + 1] down hopping matrix in column order
  uint32_t *kscol = nullptr;    // [nnz] column | (sign of JW s_c s_c') << 31
  double *kval = nullptr;       // [nnz] -t_b JW s_c s_c'
  int32_t *short_rows = nullptr;   // rows with a nontrivial stabiliser
  int n_short = 0;
  double *scratch = nullptr;    // [n_short * cols]
  unsigned long long *d_count = nullptr;
  double diag0 = 0.0;           // eps (N_up + N_dn) for uniform eps
  int fix = 0;                  // integer accumulation of the +-t hops (uniform t)
  int s0 = 0;                   // guard bits of the fixed-point terms
  double mt = 0.0;              // -t
  int *d_clean = nullptr;       // k_k0_clean's flag
};

constexpr int kDiagTab = 32;   // U n + eps (N_up + N_dn) for n = 0 .. 31 doubly occupied sites

struct K0View {
  double diag_tab[kDiagTab];
  int64_t rows, cols;
  const uint32_t *rep;
  const int32_t *per, *st_ptr, *st;
  const int32_t *uh_ptr, *uh_row, *uh_t;
  const double *uh_val;
  const uint32_t *cinfo, *cbits;
  const int32_t *tab_off;
  const uint16_t *tab;
  const int32_t *krp;
  const uint32_t *kscol;
  const double *kval;
  int g;
  int s0;
  double mt;
};

static K0View k0_view(const hub_ctx *h) {
  const K0State *k = h->k0;
  K0View v{};
  for (int n = 0; n < kDiagTab; ++n) v.diag_tab[n] = h->U0 * (double)n + k->diag0;
  v.rows = k->rows;
  v.cols = k->cols;
  v.rep = k->rep;
  v.per = k->per;
  v.st_ptr = k->st_ptr;
  v.st = k->st;
  v.uh_ptr = k->uh_ptr;
  v.uh_row = k->uh_row;
  v.uh_t = k->uh_t;
  v.uh_val = k->uh_val;
  v.cinfo = k->cinfo;
  v.cbits = k->cbits;
  v.tab_off = k->tab_off;
  v.tab = k->tab;
  v.krp = k->krp;
  v.kscol = k->kscol;
  v.kval = k->kval;
  v.g = k->g;
  v.s0 = k->s0;
  v.mt = k->mt;
  return v;
}

// ---------------------------------------------------------------------------------------
// Device side
// ---------------------------------------------------------------------------------------

// Where element e moves column c = (j, k) inside its block: the column of c_k' with
// e c_k = c_k' h', and whether sigma_j(h') = -1.
__device__ __forceinline__ uint32_t k0_move(const K0View &K, uint32_t c, uint32_t ci, int e, bool *flip) {
  const int k = (int)(ci & 0xff), type = (int)((ci >> 8) & 0xff);
  const int off = __ldg(K.tab_off + 2 * type), bs = __ldg(K.tab_off + 2 * type + 1);
  const uint32_t w = __ldg(K.tab + off + e * bs + k);
  *flip = (w & 0x8000u) != 0;
  return c - (uint32_t)k + (w & 0xffu);
}

// Row value of the product at (i, c) before the projection of short rows, FP64 throughout.
// xi: row i of x (in global memory, or staged in shared memory)
__device__ __forceinline__ double k0_row_value(const K0View &K, int64_t i, int64_t c, const double *__restrict__ x,
                                               const double *xi) {
  double acc = K.diag_tab[__popc(__ldg(K.rep + i) & __ldg(K.cbits + c))] * xi[c];
  const int k0 = __ldg(K.krp + c), k1 = __ldg(K.krp + c + 1);
  int k = k0;
  for (; k + 4 <= k1; k += 4) {          // four gathers in flight before the multiply-adds
    uint32_t w[4];
    double v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) w[j] = __ldg(K.kscol + k + j);
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = xi[w[j] & 0x7fffffffu];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc = fma(__ldg(K.kval + k + j), v[j], acc);
  }
  for (; k < k1; ++k) acc = fma(__ldg(K.kval + k), xi[__ldg(K.kscol + k) & 0x7fffffffu], acc);
  const uint32_t ci = __ldg(K.cinfo + c);
  const int h0 = __ldg(K.uh_ptr + i), h1 = __ldg(K.uh_ptr + i + 1);
  for (k = h0; k < h1; ++k) {
    bool flip;
    const uint32_t c2 = k0_move(K, (uint32_t)c, ci, __ldg(K.uh_t + k) & 0xff, &flip);
    const double cf = __ldg(K.uh_val + k);
    acc = fma(flip ? -cf : cf, x[(int64_t)__ldg(K.uh_row + k) * K.cols + c2], acc);
  }
  return acc;
}

// Signed sum of FP64 values in 64-bit fixed point (see the integer accumulation above).
struct FixSum {
  long long acc;
  int e;      // largest biased exponent so far (0: no nonzero term yet)
  int bad;    // an Inf or NaN term was seen
};

// Four terms at once: one rescale to the largest of their exponents, then four aligned adds.
// kClean: the vector holds only zeros and normal numbers (checked before the launch), so an
// exponent field of 0 marks a zero term and no term is Inf or NaN.
template <bool kClean>
__device__ __forceinline__ void fix_add4(FixSum &f, const double (&x)[4], const bool (&neg)[4], int s0) {
  int ek[4];
  unsigned long long m[4];
  int emax = f.e;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x[j]);
    ek[j] = (int)((b >> 52) & 0x7ff);
    m[j] = b & 0x000fffffffffffffull;
    if (kClean) {
      if (ek[j]) m[j] |= 0x0010000000000000ull;
    } else if (ek[j] == 0x7ff) {
      f.bad = 1;
      ek[j] = 0;
      m[j] = 0;
    } else if (ek[j] == 0) {
      ek[j] = m[j] ? 1 : 0;                 // subnormal: exponent of 2^-1022, no implicit bit
    } else {
      m[j] |= 0x0010000000000000ull;
    }
    emax = max(emax, ek[j]);
  }
  if (emax > f.e) {
    const int d = emax - f.e;
    f.acc = d >= 63 ? (f.acc < 0 ? -1ll : 0ll) : (f.acc >> d);
    f.e = emax;
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int sh = f.e - ek[j];
    const long long v = sh >= 62 ? 0ll : (long long)((m[j] << s0) >> sh);
    const bool sgn = (((unsigned long long)__double_as_longlong(x[j]) >> 63) != 0) != neg[j];
    f.acc += sgn ? -v : v;
  }
}

template <bool kClean>
__device__ __forceinline__ void fix_add(FixSum &f, double x, bool neg, int s0) {
  const double xs[4] = {x, 0.0, 0.0, 0.0};
  const bool ns[4] = {neg, false, false, false};
  fix_add4<kClean>(f, xs, ns, s0);
}

// acc * 2^(e - 1075 - s0): the power of two is built from its exponent bits, in two factors
// when it lies below the normal range (e near the bottom of the exponent range).
__device__ __forceinline__ double fix_value(const FixSum &f, int s0) {
  if (f.bad) return __longlong_as_double(0x7ff8000000000000ll);
  const int n = f.e - 1075 - s0;   // >= -1085 and <= 971
  const int n1 = n < -1022 ? -1022 : n, n2 = n - n1;
  const double p1 = __longlong_as_double((long long)(n1 + 1023) << 52);
  const double p2 = __longlong_as_double((long long)(n2 + 1023) << 52);
  return (double)f.acc * p1 * p2;
}

// Row value on the integer path: diag x + (-t) S + (hops with other coefficients, FP64).
template <bool kClean>
__device__ __forceinline__ double k0_row_value_fix(const K0View &K, int64_t i, int64_t c,
                                                    const double *__restrict__ x, const double *xi) {
  FixSum f{0ll, 0, 0};
  double side = 0.0;
  const int k0 = __ldg(K.krp + c), k1 = __ldg(K.krp + c + 1);
  int k = k0;
  for (; k + 4 <= k1; k += 4) {          // four gathers in flight before any arithmetic
    uint32_t w[4];
    double v[4];
    bool ng[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) w[j] = __ldg(K.kscol + k + j);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      v[j] = xi[w[j] & 0x7fffffffu];
      ng[j] = (w[j] >> 31) != 0;
    }
    fix_add4<kClean>(f, v, ng, K.s0);
  }
  for (; k < k1; ++k) {
    const uint32_t w = __ldg(K.kscol + k);
    fix_add<kClean>(f, xi[w & 0x7fffffffu], (w >> 31) != 0, K.s0);
  }
  const uint32_t ci = __ldg(K.cinfo + c);
  const int h0 = __ldg(K.uh_ptr + i), h1 = __ldg(K.uh_ptr + i + 1);
  for (k = h0; k + 4 <= h1; k += 4) {
    int tw[4];
    double v[4];
    bool fl[4], ng[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      tw[j] = __ldg(K.uh_t + k + j);
      const uint32_t c2 = k0_move(K, (uint32_t)c, ci, tw[j] & 0xff, &fl[j]);
      v[j] = x[(int64_t)__ldg(K.uh_row + k + j) * K.cols + c2];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      ng[j] = fl[j] != ((tw[j] & kHopNeg) != 0);
      if (!(tw[j] & kHopUnit)) {
        const double cf = __ldg(K.uh_val + k + j);
        side = fma(fl[j] ? -cf : cf, v[j], side);
        v[j] = 0.0;
      }
    }
    fix_add4<kClean>(f, v, ng, K.s0);
  }
  for (; k < h1; ++k) {
    const int tw = __ldg(K.uh_t + k);
    bool flip;
    const uint32_t c2 = k0_move(K, (uint32_t)c, ci, tw & 0xff, &flip);
    const double v = x[(int64_t)__ldg(K.uh_row + k) * K.cols + c2];
    if (tw & kHopUnit) {
      fix_add<kClean>(f, v, flip != ((tw & kHopNeg) != 0), K.s0);
    } else {
      const double cf = __ldg(K.uh_val + k);
      side = fma(flip ? -cf : cf, v, side);
    }
  }
  const double diag = K.diag_tab[__popc(__ldg(K.rep + i) & __ldg(K.cbits + c))];
  if (kClean) {
    // (-t) 2^(e - 1075 - s0) formed exactly in the exponent field of -t (a normal number for
    // every exponent of the checked vector), so one FMA gives the same rounding as
    // (-t) (acc 2^(e - 1075 - s0)); e = 0: every term was zero
    const double sc =
        f.e ? __longlong_as_double(__double_as_longlong(K.mt) + ((long long)(f.e - 1075 - K.s0) << 52)) : 0.0;
    return fma(diag, xi[c], fma(sc, (double)f.acc, side));
  }
  return fma(diag, xi[c], fma(K.mt, fix_value(f, K.s0), side));
}

template <bool kFix, bool kClean>
__device__ __forceinline__ double k0_value(const K0View &K, int64_t i, int64_t c, const double *__restrict__ x,
                                           const double *xi) {
  if (kFix) return k0_row_value_fix<kClean>(K, i, c, x, xi);
  return k0_row_value(K, i, c, x, xi);
}

// Member of the orbit of column c under the stabiliser entry s of row i: its column and the
// sign beta with X[i, c] = beta X[i, member].
__device__ __forceinline__ uint32_t k0_member(const K0View &K, int s, uint32_t c, int *sign) {
  const int w = __ldg(K.st + s);
  bool flip;
  const uint32_t pos = k0_move(K, c, __ldg(K.cinfo + c), w & 0xff, &flip);
  *sign = (((w >> 8) & 1) != 0) != flip ? -1 : 1;
  return pos;
}

// Projection of a short row onto its tied orbits at column c: the orbit's average, summed
// from its smallest member in stabiliser order, times the sign relating c to that member; 0
// for an orbit that meets itself with sign -1.  value(col) gives the unprojected entry of the
// row at a column.
template <class F>
__device__ __forceinline__ double k0_projected(const K0View &K, int64_t i, int64_t c, F value) {
  const int s0 = __ldg(K.st_ptr + i), s1 = __ldg(K.st_ptr + i + 1);
  uint32_t least = (uint32_t)c;
  int ls = 1;
  for (int s = s0; s < s1; ++s) {
    int sg;
    const uint32_t pos = k0_member(K, s, (uint32_t)c, &sg);
    if (pos == (uint32_t)c && sg < 0) return 0.0;
    if (pos < least) {
      least = pos;
      ls = sg;
    }
  }
  double sum = value((int64_t)least);
  for (int s = s0; s < s1; ++s) {
    int sg;
    const uint32_t pos = k0_member(K, s, least, &sg);
    const double v = value((int64_t)pos);
    sum += sg < 0 ? -v : v;
  }
  const double avg = sum / (double)(s1 - s0 + 1);
  return ls < 0 ? -avg : avg;
}

// gate: null, or the flag of k_k0_clean (0: the vector is clean); the kClean kernel then runs
// only on a clean vector and the other one only on a vector that is not.
template <bool kFix, bool kClean>
__global__ void __launch_bounds__(kK0Threads, 4) k_k0_apply(K0View K, const double *__restrict__ x,
                                                         double *__restrict__ y, const int *__restrict__ gate) {
  if (gate && ((__ldg(gate) == 0) != kClean)) return;
  const int64_t chunks = (K.cols + kK0Threads - 1) / kK0Threads;
  const int64_t tiles = K.rows * chunks;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t i = tile / chunks;
    const int64_t c = (tile - i * chunks) * kK0Threads + threadIdx.x;
    if (c >= K.cols) continue;
    double v;
    if (__ldg(K.st_ptr + i) == __ldg(K.st_ptr + i + 1))
      v = k0_value<kFix, kClean>(K, i, c, x, x + i * K.cols);
    else
      v = k0_projected(K, i, c, [&](int64_t col) { return k0_value<kFix, kClean>(K, i, col, x, x + i * K.cols); });
    y[i * K.cols + c] = v;
  }
}

// *flag |= 1 unless every entry of x is zero or a normal number whose exponent field lies in
// [lo, hi] (*flag zeroed before the launch)
__global__ void k_k0_clean(int64_t n, const double *__restrict__ x, int lo, int hi, int *__restrict__ flag) {
  int bad = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x[k]);
    const int e = (int)((b >> 52) & 0x7ff);
    if ((b << 1) != 0ull && (e < lo || e > hi)) bad = 1;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

// scratch[s, c] = x[short_rows[s], c]
__global__ void k_k0_gather_short(int64_t cols, int n_short, const int32_t *__restrict__ short_rows,
                                  const double *__restrict__ x, double *__restrict__ scratch) {
  const int64_t n = (int64_t)n_short * cols;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = k / cols;
    scratch[k] = x[(int64_t)short_rows[s] * cols + (k - s * cols)];
  }
}

// y[short_rows[s], c] = projection of scratch row s at c
__global__ void k_k0_project_short(K0View K, int n_short, const int32_t *__restrict__ short_rows,
                                   const double *__restrict__ scratch, double *__restrict__ y) {
  const int64_t n = (int64_t)n_short * K.cols;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = k / K.cols, c = k - s * K.cols;
    const double *src = scratch + s * K.cols;
    const int64_t i = short_rows[s];
    y[i * K.cols + c] = k0_projected(K, i, c, [&](int64_t col) { return src[col]; });
  }
}

// Number of states of the sector in the short rows: columns that are the smallest member of
// an orbit that does not meet itself with sign -1.
__global__ void k_k0_count_short(K0View K, int n_short, const int32_t *__restrict__ short_rows,
                                 unsigned long long *__restrict__ count) {
  const int64_t n = (int64_t)n_short * K.cols;
  unsigned long long mine = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = k / K.cols, c = k - s * K.cols;
    const int64_t i = short_rows[s];
    bool least = true, null = false;
    for (int e = K.st_ptr[i]; e < K.st_ptr[i + 1]; ++e) {
      int sg;
      const uint32_t pos = k0_member(K, e, (uint32_t)c, &sg);
      if (pos < (uint32_t)c) least = false;
      if (pos == (uint32_t)c && sg < 0) null = true;
    }
    if (least && !null) ++mine;
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(count, mine);
}

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------

void k0_release(hub_ctx *h) {
  K0State *k = h->k0;
  if (!k) return;
  dev_free(k->rep);
  dev_free(k->per);
  dev_free(k->st_ptr);
  dev_free(k->st);
  dev_free(k->uh_ptr);
  dev_free(k->uh_row);
  dev_free(k->uh_t);
  dev_free(k->uh_val);
  dev_free(k->cinfo);
  dev_free(k->cbits);
  dev_free(k->tab_off);
  dev_free(k->tab);
  dev_free(k->krp);
  dev_free(k->kscol);
  dev_free(k->kval);
  dev_free(k->short_rows);
  dev_free(k->scratch);
  dev_free(k->d_count);
  dev_free(k->d_clean);
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

// H must commute with every generator: each bond moved by it is a bond with the same t, and U
// and eps are the same on every site.
static int check_invariant(const hub_ctx *h, int n_gen, const int32_t *perms) {
  std::map<std::pair<int, int>, double> bonds;
  for (int b = 0; b < h->n_bonds; ++b) {
    const int i = h->bonds[2 * b], j = h->bonds[2 * b + 1];
    bonds[{std::min(i, j), std::max(i, j)}] = h->t[b];
  }
  for (int a = 0; a < n_gen; ++a)
    for (int b = 0; b < h->n_bonds; ++b) {
      const int i = perms[a * h->M + h->bonds[2 * b]], j = perms[a * h->M + h->bonds[2 * b + 1]];
      const auto it = bonds.find({std::min(i, j), std::max(i, j)});
      if (it == bonds.end() || it->second != h->t[b])
        return fail(HUB_ERR_ARG, "hub_set_symmetry: the bonds are not invariant under the translations");
    }
  if (!h->uniform_U) return fail(HUB_ERR_ARG, "hub_set_symmetry: U differs between sites");
  for (int i = 1; i < h->M; ++i)
    if (h->eps[i] != h->eps[0]) return fail(HUB_ERR_ARG, "hub_set_symmetry: eps differs between sites");
  return HUB_OK;
}

// Device copy of a host table: HUB_ERR_OOM if the allocation fails, HUB_ERR_CUDA if the copy does.
template <class T>
static int upload(T **dst, const std::vector<T> &src, const char *what) {
  if (!dev_alloc((void **)dst, sizeof(T) * std::max<size_t>(src.size(), 1), what)) return HUB_ERR_OOM;
  if (!src.empty()) HUB_CUDA(cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
  return HUB_OK;
}

static int k0_build(hub_ctx *h, const Group &G) {
  const int M = h->M, Nu = h->N[0], Nd = h->N[1], g = G.g;
  K0State *k = new (std::nothrow) K0State();
  if (!k) return fail(HUB_ERR_OOM, "hub_set_symmetry: host allocation failed");
  h->k0 = k;
  k->g = g;
  k->cols = h->count[1];
  k->diag0 = (h->eps.empty() ? 0.0 : h->eps[0]) * (double)(Nu + Nd);

  // every orbit has at most |G| members, so rows >= count_up / |G|: refuse before enumerating
  // when even that many rows of one vector cannot fit
  size_t free_b = 0, total_b = 0;
  HUB_CUDA(cudaMemGetInfo(&free_b, &total_b));
  if (8.0 * ((double)h->count[0] / g) * (double)k->cols > (double)free_b)
    return fail(HUB_ERR_OOM, "hub_set_symmetry: one vector of the sector does not fit");

  // rows: up representatives, ascending, orbit sizes, stabiliser lists
  std::vector<uint32_t> reps;
  std::vector<int32_t> per, st_ptr(1, 0), st;
  for (uint32_t x : strings_of(M, Nu)) {
    const OrbitOf o = orbit_of(G, x);
    if (o.least != x) continue;
    reps.push_back(x);
    per.push_back(g / (int)o.stab.size());
    for (const auto &hs : o.stab)
      if (hs.first != 0) st.push_back(hs.first | ((G.chi[hs.first] * hs.second < 0) ? (1 << 8) : 0));
    st_ptr.push_back((int32_t)st.size());
  }
  k->rows = (int64_t)reps.size();
  k->rep_h = reps;
  k->per_h = per;
  if (8.0 * (double)k->rows * (double)k->cols > (double)free_b)
    return fail(HUB_ERR_OOM, "hub_set_symmetry: one vector of the sector does not fit");

  // integer accumulation: uniform nonzero t and room for every entry's terms (at most one per
  // bond and spin) with at least one guard bit: terms * 2^(53 + s0) < 2^63
  const Ham Hv = h->view();
  int terms_log2 = 0;
  while ((1 << terms_log2) < 2 * std::max(h->n_bonds, 1)) ++terms_log2;
  k->s0 = 10 - terms_log2;
  k->mt = -Hv.t0;
  k->fix = (Hv.uniform_t && Hv.t0 != 0.0 && k->s0 >= 1) ? 1 : 0;

  // up-hop lists: hopped string u', its representative R_i' and the first element e0 with
  // e0 |u'> = s |R_i'>, so that g = e0^-1 maps R_i' to s u' and the gather moves by g^-1 = e0
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
      const OrbitOf o = orbit_of(G, u2);
      const auto it = std::lower_bound(reps.begin(), reps.end(), o.least);
      if (it == reps.end() || *it != o.least) return fail(HUB_ERR_CUDA, "hub_set_symmetry: representative not found");
      const int i2 = (int)(it - reps.begin());
      const int e0 = o.e_least, s = o.s_least;
      const double cf = val * s * G.chi[G.inv[e0]];
      int tw = e0;
      if (per[i] == per[i2] && k->fix) {
        tw |= kHopUnit;
        if (cf / k->mt < 0) tw |= kHopNeg;
      }
      uh_row.push_back(i2);
      uh_t.push_back(tw);
      uh_val.push_back(cf * std::sqrt((double)per[i] / (double)per[i2]));
    }
    uh_ptr.push_back((int32_t)uh_row.size());
  }
  std::vector<int32_t> shorts;
  for (size_t i = 0; i < reps.size(); ++i)
    if (st_ptr[i + 1] > st_ptr[i]) shorts.push_back((int32_t)i);
  k->n_short = (int)shorts.size();

  // columns in the order of Table I (down representatives ascending, each followed by the rest
  // of its orbit) and one move table per stabiliser type
  const std::vector<uint32_t> dn = strings_of(M, Nd);
  if ((int64_t)dn.size() != k->cols) return fail(HUB_ERR_CUDA, "hub_set_symmetry: down basis size mismatch");
  Columns C;
  std::string cerr;
  if (build_columns(G, dn, &C, &cerr)) return fail(HUB_ERR_ARG, "hub_set_symmetry: " + cerr);
  const std::vector<uint32_t> &cinfo = C.cinfo, &cbits = C.cbits;
  const std::vector<int32_t> &csign = C.csign, &pos = C.pos, &tab_off = C.tab_off;
  const std::vector<uint16_t> &tab = C.tab;
  k->col_bits_h = cbits;
  k->col_sign_h = csign;

  // the down hopping matrix of a2 relabelled to this column order, signs s_c s_c' folded in
  const SpinCSR &cd = h->csr[h->shared ? 0 : 1];
  std::vector<int32_t> rp(k->cols + 1), col(std::max<int64_t>(cd.nnz, 1));
  std::vector<uint32_t> scol(std::max<int64_t>(cd.nnz, 1));
  std::vector<double> val(std::max<int64_t>(cd.nnz, 1));
  HUB_CUDA(cudaMemcpy(rp.data(), cd.rowptr, sizeof(int32_t) * (k->cols + 1), cudaMemcpyDeviceToHost));
  if (cd.nnz) {
    HUB_CUDA(cudaMemcpy(col.data(), cd.col, sizeof(int32_t) * cd.nnz, cudaMemcpyDeviceToHost));
    HUB_CUDA(cudaMemcpy(scol.data(), cd.scol, sizeof(uint32_t) * cd.nnz, cudaMemcpyDeviceToHost));
    HUB_CUDA(cudaMemcpy(val.data(), cd.val, sizeof(double) * cd.nnz, cudaMemcpyDeviceToHost));
  }
  std::vector<int32_t> krp(1, 0);
  std::vector<uint32_t> kscol;
  std::vector<double> kval;
  kscol.reserve(std::max<int64_t>(cd.nnz, 1));
  kval.reserve(std::max<int64_t>(cd.nnz, 1));
  for (int64_t c = 0; c < k->cols; ++c) {
    const size_t r = (size_t)(std::lower_bound(dn.begin(), dn.end(), cbits[c]) - dn.begin());
    for (int32_t e = rp[r]; e < rp[r + 1]; ++e) {
      const int32_t c2 = pos[col[e]];
      const int sg = csign[c] * csign[c2];
      const bool neg = ((scol[e] >> 31) != 0) != (sg < 0);
      kscol.push_back((uint32_t)c2 | (neg ? 0x80000000u : 0u));
      kval.push_back(val[e] * sg);
    }
    krp.push_back((int32_t)kscol.size());
  }

  int rc = HUB_OK;
  if ((rc = upload(&k->rep, reps, "sector representatives")) || (rc = upload(&k->per, per, "sector orbits")) ||
      (rc = upload(&k->st_ptr, st_ptr, "sector stabilisers")) || (rc = upload(&k->st, st, "sector stabilisers")) ||
      (rc = upload(&k->uh_ptr, uh_ptr, "sector up hops")) || (rc = upload(&k->uh_row, uh_row, "sector up hops")) ||
      (rc = upload(&k->uh_t, uh_t, "sector up hops")) || (rc = upload(&k->uh_val, uh_val, "sector up hops")) ||
      (rc = upload(&k->cinfo, cinfo, "sector columns")) || (rc = upload(&k->cbits, cbits, "sector columns")) ||
      (rc = upload(&k->tab_off, tab_off, "sector move tables")) || (rc = upload(&k->tab, tab, "sector move tables")) ||
      (rc = upload(&k->krp, krp, "sector down hops")) || (rc = upload(&k->kscol, kscol, "sector down hops")) ||
      (rc = upload(&k->kval, kval, "sector down hops")) || (rc = upload(&k->short_rows, shorts, "sector short rows")))
    return rc;
  if (!dev_alloc((void **)&k->scratch, sizeof(double) * std::max<int64_t>(k->n_short * k->cols, 1), "sector scratch") ||
      !dev_alloc((void **)&k->d_count, sizeof(unsigned long long), "sector counter"))
    return HUB_ERR_OOM;

  // dimension: free rows count fully, short rows by their orbits
  k->dim = (k->rows - k->n_short) * k->cols;
  if (k->n_short && k->cols) {
    HUB_CUDA(cudaMemset(k->d_count, 0, sizeof(unsigned long long)));
    const int64_t n = (int64_t)k->n_short * k->cols;
    k_k0_count_short<<<(int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 32), 256>>>(
        k0_view(h), k->n_short, k->short_rows, k->d_count);
    HUB_LAUNCH_CHECK();
    unsigned long long c = 0;
    HUB_CUDA(cudaMemcpy(&c, k->d_count, sizeof(c), cudaMemcpyDeviceToHost));
    k->dim += (int64_t)c;
  }
  HUB_CUDA(cudaDeviceSynchronize());
  return HUB_OK;
}

// Launch one product kernel: CTAs of 256 columns of one row, grid-stride over rows x chunks.
template <bool kFix, bool kClean>
static int k0_launch(const hub_ctx *h, const double *x, double *y, const int *gate, cudaStream_t s) {
  const K0State *k = h->k0;
  const int64_t tiles = k->rows * ((k->cols + kK0Threads - 1) / kK0Threads);
  const int grid = (int)std::min<int64_t>(tiles, (int64_t)num_sms() * 16);
  k_k0_apply<kFix, kClean><<<grid, kK0Threads, 0, s>>>(k0_view(h), x, y, gate);
  HUB_LAUNCH_CHECK();
  return HUB_OK;
}

int k0_apply(hub_ctx *h, const double *x, double *y, cudaStream_t s) {
  const K0State *k = h->k0;
  if (k->rows == 0 || k->cols == 0) return HUB_OK;
  int rc;
  if (k->fix && h->mode == HUB_MODE_AUTO) {
    // the integer path without the Inf / NaN / subnormal handling when x holds none and every
    // scale (-t) 2^(e - 1075 - s0) of an entry exponent e is a normal number
    unsigned long long mt_bits;
    std::memcpy(&mt_bits, &k->mt, sizeof mt_bits);
    const int et = (int)((mt_bits >> 52) & 0x7ff);
    const int lo = std::max(1, 1076 + k->s0 - et), hi = std::min(2046, 2046 + 1075 + k->s0 - et);
    if (!k->d_clean && !dev_alloc((void **)&k->d_clean, sizeof(int), "momentum-sector flag")) return HUB_ERR_OOM;
    const int64_t n = k->rows * k->cols;
    count_launch(h, 3);
    HUB_CUDA(cudaMemsetAsync(k->d_clean, 0, sizeof(int), s));
    k_k0_clean<<<(int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8), 256, 0, s>>>(n, x, lo, hi,
                                                                                               k->d_clean);
    HUB_LAUNCH_CHECK();
    if ((rc = k0_launch<true, true>(h, x, y, k->d_clean, s))) return rc;
    return k0_launch<true, false>(h, x, y, k->d_clean, s);
  }
  count_launch(h);
  return k0_launch<false, false>(h, x, y, nullptr, s);
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

// Validate the generators, build the group and the tables of its sector.
static int set_translations(hub_t h, int n_gen, const int32_t *perms, const int32_t *chars, const char *who) {
  int rc = ready(h, who);
  if (rc) return rc;
  const int M = h->M;
  if (n_gen < 1 || n_gen > 8 || !perms || !chars) return fail(HUB_ERR_ARG, std::string(who) + ": bad argument");
  for (int a = 0; a < n_gen; ++a) {
    std::vector<int> hit(M, 0);
    for (int i = 0; i < M; ++i) {
      const int p = perms[a * M + i];
      if (p < 0 || p >= M || hit[p]++) return fail(HUB_ERR_ARG, std::string(who) + ": a generator is not a permutation of the sites");
    }
    if (chars[a] != 1 && chars[a] != -1) return fail(HUB_ERR_ARG, std::string(who) + ": characters must be +1 or -1");
  }
  if ((rc = check_invariant(h, n_gen, perms))) return rc;
  Group G;
  std::string err;
  if (make_group(M, n_gen, perms, chars, &G, &err)) return fail(HUB_ERR_ARG, std::string(who) + ": " + err);
  k0_release(h);
  release_vectors(h);
  rc = k0_build(h, G);
  if (rc) k0_release(h);
  return rc;
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
  if (sym == HUB_SYM_KPI && (h->M & 1)) return fail(HUB_ERR_ARG, "hub_set_symmetry: k = pi needs an even M");
  std::vector<int32_t> perm(h->M);
  for (int i = 0; i < h->M; ++i) perm[i] = (i + h->M - 1) % h->M;   // T: site i -> i - 1
  const int32_t chi = sym == HUB_SYM_KPI ? -1 : 1;
  return set_translations(h, 1, perm.data(), &chi, "hub_set_symmetry");
}

extern "C" int hub_set_translations(hub_t h, int n_gen, const int32_t *perm_host, const int32_t *char_host) {
  if (!h) return fail(HUB_ERR_ARG, "hub_set_translations: NULL handle");
  return set_translations(h, n_gen, perm_host, char_host, "hub_set_translations");
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

extern "C" int hub_k_columns(hub_t h, uint32_t *dn_host, int32_t *sign_host) {
  if (!h) return fail(HUB_ERR_ARG, "hub_k_columns: NULL handle");
  if (!h->k0) return fail(HUB_ERR_STATE, "hub_k_columns: no momentum sector is active (hub_set_symmetry)");
  const K0State *k = h->k0;
  for (int64_t c = 0; c < k->cols; ++c) {
    if (dn_host) dn_host[c] = k->col_bits_h[c];
    if (sign_host) sign_host[c] = k->col_sign_h[c];
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
