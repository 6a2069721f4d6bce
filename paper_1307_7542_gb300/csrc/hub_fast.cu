// hub_fast.cu -- the fast apply for uniform hopping (K3 fast path) and the double-float
// Lanczos built on it.
//
// The product is Eq. 11 of Sec. IV.A on the count_dn x count_up state matrix X (Eq.
// count2):  Y = X H_up^T + H_dn X + diag o X, with every hopping element -t * esign
// (Eq. 8) and diag = U popcount(I_up & I_dn) + eps(I_up) + eps(I_dn) (Sec. III.B).  The
// two hopping terms want different memory orders, so they run as two passes:
//
//   pass 1 (k_up): a CTA takes two rows (d0, d1) of X at a time.  Both rows are copied
//     whole into shared memory by bulk asynchronous copies (cp.async.bulk, completion on
//     an mbarrier), then each thread sums the H_up row of its column u for both rows from
//     shared memory (in-row gather) and adds the diagonal:
//     Z[d][u] = t S_up + diag X[d][u].
//   pass 2 (k_dn): tiles of 32 rows x 64 columns, launched strip-major (all tiles of one
//     column strip are adjacent in the grid), so the strip of X that the H_dn rows
//     combine -- count_dn x 64 values -- stays in L2 while the whole strip is processed
//     and X is read from HBM about once.  Each warp adds t S_dn to Z for its rows with
//     64-bit loads of whole rows of the strip.
//
// Vectors are double-float (hub_df.cuh), stored planar per row: row d of a vector is 2 ld
// floats, the ld high parts followed by the ld low parts (ld >= count_up, a multiple of 4,
// padding columns zero).  Both planes of a row start on 16-byte boundaries (bulk copies),
// and the two values a packed FP32x2 instruction combines always sit in adjacent words:
// (hi of row d0, hi of row d1) come from two 32-bit shared loads in pass 1, and the
// (hi, hi) / (lo, lo) pairs of columns u, u+1 from two 64-bit loads in pass 2, so no
// register shuffling is needed around the TwoSum chains.  Inside this file the columns of X
// are kept in "slot" order: spin-up states sorted by the lengths of their two hopping
// groups, so that the 32 rows of H_up a warp sums in pass 1 have nearly equal lengths
// (little divergence) while its loads and stores stay contiguous.  Pass 2 combines whole
// rows and does not care about column order.  Only the FP64 <-> double-float conversions
// at the boundary of this file map slots back to ranks.  The hopping rows are reordered by
// sign (entries adding x first, then entries subtracting x), so no per-term sign handling
// is needed, and columns are stored as uint16 when count <= 65536.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "hub_df.cuh"
#include "hub_internal.cuh"

namespace hub {

int ready(const hub_ctx *h, const char *who);
std::vector<double> tridiag_vector(const double *a, const double *b, int k, double lam);

// ---------------------------------------------------------------------------------------
// Small PTX wrappers: mbarrier and bulk copy (sm_90+).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after ~2^24 polls (each poll may suspend the thread briefly).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase) {
  for (uint32_t it = 0; it < (1u << 24); ++it)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

// ---------------------------------------------------------------------------------------
// Fast-path view (passed by value).
// ---------------------------------------------------------------------------------------
struct FastView {
  int64_t n_up, n_dn, ld;            // ld: plane length of a row (multiple of 4); row stride 2 ld
  const uint32_t *basis_up, *basis_dn;
  const int32_t *rp_up, *sp_up;      // row start and sign split of H_up
  const int32_t *rp_dn, *sp_dn;
  const void *col_up, *col_dn;       // uint16 or uint32 columns
  // H_up in sliced column-major form for pass 1.  Rows are placed in slots ordered by their
  // (add, sub) group lengths so that the 32 rows a warp handles have nearly equal lengths;
  // slot k holds row slot_row[k].  Each slice of 32 slots has, per group, a schedule of
  // steps: in one step every lane reads at most one of its entries, chosen so that at most
  // two lanes of the warp hit the same shared-memory bank (column mod 32).  A word holds the
  // columns of two steps (uint16) or one (uint32); the words of a slice are stored in
  // batches of four per lane, word i of batch b of slot k at off[k/32] + (b*32 + k%32)*4 + i,
  // so that one 16-byte load brings a lane 8 (uint16) or 4 (uint32) steps.  Idle steps
  // (schedule gaps, padding of the last word and batch) name a zero column (staged rows) or
  // the sentinel 0xffff / 0xffffffff (rows read through L2).
  const uint32_t *sl_add, *sl_sub;   // packed words
  const int32_t *sl_off_add, *sl_off_sub;
  const uint16_t *steps_add, *steps_sub;   // per slice: scheduled steps (entries per lane)
  uint32_t idle_word;                // a column word whose entries are all idle steps
  const int32_t *slot_row;           // spin-up rank held by slot k
  const uint32_t *basis_up_slot;     // spin-up strings in slot order
  int t_neg;                         // the kernels apply H / |t|: hopping sign(t), diagonal U k / |t|
  float2 Utab[32];                   // (U / |t|) k for k = popcount(I_up & I_dn)
  int *err;                          // device error flag (bounded waits)
  int fail_waits;                    // test hook: take the given-up-wait exit once the copies landed
};

template <typename Col>
__device__ __forceinline__ uint32_t colat(const void *c, int64_t k) {
  return (uint32_t)((const Col *)c)[k];
}

// ---------------------------------------------------------------------------------------
// Sign-split CSR: per row, entries with esign = -1 (element +t: add x) first, then the
// entries with esign = +1 (element -t: subtract x); columns ascending inside each group.
// ---------------------------------------------------------------------------------------
template <typename Col>
__global__ void k_split_csr(int64_t n, const int32_t *__restrict__ rp, const uint32_t *__restrict__ scol,
                            int32_t *__restrict__ sp, Col *__restrict__ col) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = rp[r], b = rp[r + 1];
    int32_t w = a;
    for (int32_t k = a; k < b; ++k)
      if (scol[k] >> 31) col[w++] = (Col)(scol[k] & 0x7fffffffu);
    sp[r] = w;
    for (int32_t k = a; k < b; ++k)
      if (!(scol[k] >> 31)) col[w++] = (Col)(scol[k] & 0x7fffffffu);
  }
}

// basis of the spin-up states in slot order
__global__ void k_to_slots(int64_t n, const int32_t *__restrict__ slot_row, const uint32_t *__restrict__ basis,
                           uint32_t *__restrict__ basis_slot) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    basis_slot[k] = basis[slot_row[k]];
}

// ---------------------------------------------------------------------------------------
// Conversions between the ABI's FP64 layout (row length n_up, rank order) and the planar
// double-float layout (slot order), with a power-of-two scale.
// ---------------------------------------------------------------------------------------
// The fast path holds a vector as double-floats scaled by 2^-shift, max |x| 2^-shift in
// [1, 2).  Its per-entry error bound (about 20 u^2 (|H||x|)_n, u = 2^-24) needs every
// term, product and sum it forms to keep 48 bits, i.e. FP32 low parts above the FP32
// subnormal range: with nonzero |x| 2^-shift >= 2^-80 and a diagonal coefficient U / |t|
// of 0 or in [2^-16, 2^16] (fast_eligible), every nonzero product is at least 2^-96, its
// low part at least 2^-120.  The scaled results must also map back into the FP64 range.
// The window:
// the largest biased FP64 exponent in [kExpLo, kExpHi] and every nonzero entry's exponent
// at most kExpSpan below it; FP64 subnormals, infinities and NaN are outside.  A vector
// outside the window is multiplied by the FP64 kernel instead.
constexpr int kExpSpan = 80, kExpLo = 200, kExpHi = 1900;

// partials[block] = largest biased FP64 exponent of the block's elements (2047 for inf or
// NaN), partials[nblk + block] = smallest biased exponent among its nonzero elements (0 for
// an FP64 subnormal, 2048 if all are zero); nblk = gridDim.x
__global__ void k_exp_range(int64_t D, const double *__restrict__ x, int *__restrict__ partials) {
  int m = 0, n = 2048;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < D; k += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t b = (uint64_t)__double_as_longlong(x[k]);
    const int e = (int)((b >> 52) & 0x7ffu);
    m = max(m, e);
    if (b << 1) n = min(n, e);
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    n = min(n, __shfl_xor_sync(0xffffffffu, n, o));
  }
  __shared__ int wm[32], wn[32];
  if ((threadIdx.x & 31) == 0) {
    wm[threadIdx.x >> 5] = m;
    wn[threadIdx.x >> 5] = n;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool in = threadIdx.x < (blockDim.x >> 5);
    int a = in ? wm[threadIdx.x] : 0, c = in ? wn[threadIdx.x] : 2048;
    for (int o = 16; o > 0; o >>= 1) {
      a = max(a, __shfl_xor_sync(0xffffffffu, a, o));
      c = min(c, __shfl_xor_sync(0xffffffffu, c, o));
    }
    if (threadIdx.x == 0) {
      partials[blockIdx.x] = a;
      partials[gridDim.x + blockIdx.x] = c;
    }
  }
}

// Range of partials[0 .. nblk) (stride: nblk to the minima, as k_exp_range writes them;
// n_sets such sets back to back).
__device__ __forceinline__ void range_of(const int *__restrict__ p, int nblk, int n_sets, int &emax, int &emin) {
  int a = 0, c = 2048;
  for (int s = 0; s < n_sets; ++s)
    for (int k = threadIdx.x; k < nblk; k += blockDim.x) {
      a = max(a, p[2 * s * nblk + k]);
      c = min(c, p[(2 * s + 1) * nblk + k]);
    }
  for (int o = 16; o > 0; o >>= 1) {
    a = max(a, __shfl_xor_sync(0xffffffffu, a, o));
    c = min(c, __shfl_xor_sync(0xffffffffu, c, o));
  }
  __shared__ int wa[32], wc[32];
  if ((threadIdx.x & 31) == 0) {
    wa[threadIdx.x >> 5] = a;
    wc[threadIdx.x >> 5] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a = max(a, wa[k]);
      c = min(c, wc[k]);
    }
    emax = a;
    emin = c;
  }
}

__device__ __forceinline__ bool out_of_window(int emax, int emin) {
  return emax != 0 && (emax < kExpLo || emax > kExpHi || emin < emax - kExpSpan);
}

// One block: scale[0] = shift (max |x| 2^-shift in [1, 2); 0 for a zero vector), scale[1] =
// 1 if the vector lies outside the fast path's window (see kExpSpan).
__global__ void k_scale(const int *__restrict__ partials, int nblk, int *__restrict__ scale) {
  int emax = 0, emin = 2048;
  range_of(partials, nblk, 1, emax, emin);
  if (threadIdx.x == 0) {
    scale[0] = emax == 0 ? 0 : emax - 1023;
    scale[1] = out_of_window(emax, emin) ? 1 : 0;
  }
}

// Host-buffer product, after all chunks: n_sets exponent partial sets (one per chunk, the
// first one gave the scale used so far).  scale[2] = shift of the whole vector, scale[3] =
// its window flag; flag[0] = 2 if the whole vector lies outside the window, 1 if its
// largest exponent exceeds the first chunk's (convert again with scale[2]), else 0.
__global__ void k_scale_all(const int *__restrict__ partials, int nblk, int n_sets, int *__restrict__ scale,
                            int *__restrict__ flag) {
  int emax = 0, emin = 2048;
  range_of(partials, nblk, n_sets, emax, emin);
  if (threadIdx.x == 0) {
    const int shift = emax == 0 ? 0 : emax - 1023;
    const bool out = out_of_window(emax, emin);
    scale[2] = shift;
    scale[3] = out ? 1 : 0;
    flag[0] = out ? 2 : (shift != scale[0] ? 1 : 0);
  }
}

// out (planar, slot order) = 2^-shift x (FP64, rank order) for rows r0 .. r1 - 1, shift =
// scale[0] (0 when scale is null); one row per block and step
__global__ void k_f64_to_df(int64_t r0, int64_t r1, int64_t n_up, int64_t ld, const double *__restrict__ x,
                            const int *__restrict__ scale, const int32_t *__restrict__ slot_row,
                            float *__restrict__ out) {
  const int shift = scale ? scale[0] : 0;
  for (int64_t d = r0 + blockIdx.x; d < r1; d += gridDim.x) {
    float *__restrict__ row = out + d * 2 * ld;
    const double *__restrict__ xr = x + d * n_up;
    for (int64_t u = threadIdx.x; u < ld; u += blockDim.x) {
      const float2 v = u < n_up ? f64_to_df(xr[slot_row[u]], shift) : make_float2(0.f, 0.f);
      row[u] = v.x;
      row[ld + u] = v.y;
    }
  }
}

// y[d][u] (FP64, rank order) = tabs 2^shift v[d][slot_of[u]] (planar double-float, slot
// order) for rows r0 .. r1 - 1, shift = scale[0]; one row per block and step so that the
// gathers of a row are served from L1.  Nothing is written when scale[1] is set (the FP64
// kernel writes y instead).  tabs = |t|: the kernels applied H / |t|.
__global__ void k_unpermute(int64_t r0, int64_t r1, int64_t n_up, int64_t ld, const float *__restrict__ v,
                            const int32_t *__restrict__ slot_of, const int *__restrict__ scale, double tabs,
                            double *__restrict__ y) {
  if (scale[1]) return;
  const int shift = scale[0];
  for (int64_t d = r0 + blockIdx.x; d < r1; d += gridDim.x) {
    const float *__restrict__ row = v + d * 2 * ld;
    for (int64_t u = threadIdx.x; u < n_up; u += blockDim.x) {
      const int32_t s = slot_of[u];
      const double val = df_to_f64(make_float2(row[s], row[ld + s]), shift);
      y[d * n_up + u] = tabs == 1.0 ? val : val * tabs;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Pass 1: spin-up hops (in-row gather from shared memory) and the diagonal.  A CTA takes
// two rows (d0, d1) at a time: their four planes are staged (four bulk copies completing on
// one mbarrier), every column index is loaded once for both rows, and the two rows' TwoSum
// chains run as one packed FP32x2 chain.  While a pair is computed, the CTA's next pair is
// prefetched into L2.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Staged planes: hi(d0), lo(d0), hi(d1), lo(d1) at k * kUpPlane floats (compile-time
// offsets, so the four loads of a term share one address; kUpPlane is a multiple of 32, so
// all planes have the same bank alignment).  Entries ld and ld + 1 of every plane are zero
// and serve as the column of idle schedule steps (adding zero is exact).
constexpr int kUpPlane = 14080;

// FP64 value of lane a + lane b of a packed (hi, lo) pair
__device__ __forceinline__ double df2_lanes_to_f64(f2x h, f2x l) {
  const float2 hh = upk2(h), ll = upk2(l);
  return df_to_f64(make_float2(hh.x, ll.x), 0) + df_to_f64(make_float2(hh.y, ll.y), 0);
}

// The Lanczos recurrence fused into pass 1 (kUpd): the staged rows are those of w (the
// previous step's pass-2 output); before the gathers each CTA forms r_j = w + c r_{j-1}
// (c = -alpha_{j-1} / |r_{j-1}|, the update of Sec. IV's recurrence) in shared memory, writes
// it back over w in HBM for pass 2 and the next steps, and accumulates |r_j|^2.
#ifndef HUB_UPD_Q
#define HUB_UPD_Q 1   // column quads per thread whose loads the fused update issues together
#endif
#ifndef HUB_FUSED_UPDATE
#define HUB_FUSED_UPDATE 1   // 0: the Lanczos update as a separate vector pass before pass 1
#endif
#ifndef HUB_UP_PAIRED
#define HUB_UP_PAIRED 1   // 1: pass 1 sums with DfSumP (low parts of a word's two entries paired); 0: DfSum4
#endif
#ifndef HUB_UP_THREADS
#define HUB_UP_THREADS 1024   // threads of the pass-1 CTA (one CTA per SM; fewer leave more registers)
#endif
constexpr int kUpThreads = HUB_UP_THREADS;
static_assert(kUpThreads % 32 == 0 && kUpThreads >= 512 && kUpThreads <= 1024, "pass-1 CTA size");
constexpr int kUpdQ = HUB_UPD_Q;
// Lanczos steps per host read-back for sectors of at most kBatchStepsMaxDim states
constexpr int kMaxBatchSteps = 8;
constexpr int64_t kBatchStepsMaxDim = 1 << 21;
constexpr bool kFusedUpdate = HUB_FUSED_UPDATE != 0;

struct UpdArgs {
  const float *r_prev;               // r_{j-1} (planar rows)
  const float2 *coef;                // coef[2] = c (double-float)
  double *partials;                  // |r_j|^2 per CTA
};

template <typename Col, bool kUpd>
__global__ void __launch_bounds__(kUpThreads, 1) k_up(const FastView F, float *x, float *__restrict__ z,
                                                int64_t p_begin, int64_t p_end, UpdArgs U) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float *xs = reinterpret_cast<float *>(smem_raw);
  __shared__ __align__(8) uint64_t bar;
  __shared__ float2 utab[32];
  const int tid = threadIdx.x;
  const int64_t ld = F.ld;
  const uint32_t pbytes = (uint32_t)(ld * sizeof(float));
  if (tid < 32) utab[tid] = F.Utab[tid];
  if (tid < 8) xs[(tid >> 1) * kUpPlane + ld + (tid & 1)] = 0.f;
  __shared__ double wnorm[32];              // |r_j|^2 per warp, summed in a fixed order (kUpd)
  if (kUpd && tid < 32) wnorm[tid] = 0.0;
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  for (int64_t p = p_begin + blockIdx.x; p < p_end; p += gridDim.x) {   // row pairs p_begin .. p_end - 1
    const int64_t d0 = 2 * p, d1 = (2 * p + 1 < F.n_dn) ? 2 * p + 1 : 2 * p;   // odd tail: same row twice
    if (tid == 0) {
      const float *r0 = x + d0 * 2 * ld, *r1 = x + d1 * 2 * ld;
      fence_proxy_async();
      mbar_expect_tx(&bar, 4 * pbytes);
      bulk_g2s(xs, r0, pbytes, &bar);
      bulk_g2s(xs + kUpPlane, r0 + ld, pbytes, &bar);
      bulk_g2s(xs + 2 * kUpPlane, r1, pbytes, &bar);
      bulk_g2s(xs + 3 * kUpPlane, r1 + ld, pbytes, &bar);
      const int64_t pn = p + gridDim.x;
      if (pn < p_end) {
        prefetch_l2(x + 2 * pn * 2 * ld, 2 * pbytes);
        if (2 * pn + 1 < F.n_dn) prefetch_l2(x + (2 * pn + 1) * 2 * ld, 2 * pbytes);
        if (kUpd) {
          prefetch_l2(U.r_prev + 2 * pn * 2 * ld, 2 * pbytes);
          if (2 * pn + 1 < F.n_dn) prefetch_l2(U.r_prev + (2 * pn + 1) * 2 * ld, 2 * pbytes);
        }
      }
    }
    if (!mbar_wait_bounded(&bar, phase)) {
      if (tid == 0) atomicExch(F.err, 1);
      mbar_wait_bounded(&bar, phase);      // give a late copy one more bounded chance to land
      return;
    }
    if (F.fail_waits) {                    // test hook: the same exit, after the copies landed
      if (tid == 0) atomicExch(F.err, 1);
      return;
    }
    phase ^= 1u;
    if (kUpd) {
      // r_j = w + c r_{j-1} for both rows, four columns per thread step: in shared memory,
      // in HBM over w, and into |r_j|^2 (lane b counted only when the rows differ)
      const float *pr0 = U.r_prev + d0 * 2 * ld, *pr1 = U.r_prev + d1 * 2 * ld;
      float *x0 = x + d0 * 2 * ld, *x1 = x + d1 * 2 * ld;
      const float2 cf = U.coef[2];
      const f2x cph = bcast2(cf.x), cpl = bcast2(cf.y);
      DfAcc2 nacc{0ull, 0ull};
      // kUpdQ quads per thread and batch, their global loads issued before any arithmetic
      const int64_t stride = 4 * (int64_t)blockDim.x;
      for (int64_t q0 = 4 * (int64_t)tid; q0 < ld; q0 += kUpdQ * stride) {
        float4 ph0[kUpdQ], pl0[kUpdQ], ph1[kUpdQ], pl1[kUpdQ];
#pragma unroll
        for (int i = 0; i < kUpdQ; ++i) {
          const int64_t q = q0 + i * stride;
          if (q < ld) {
            ph0[i] = *reinterpret_cast<const float4 *>(pr0 + q);
            pl0[i] = *reinterpret_cast<const float4 *>(pr0 + ld + q);
            ph1[i] = *reinterpret_cast<const float4 *>(pr1 + q);
            pl1[i] = *reinterpret_cast<const float4 *>(pr1 + ld + q);
          }
        }
#pragma unroll
        for (int i = 0; i < kUpdQ; ++i) {
          const int64_t q = q0 + i * stride;
          if (q >= ld) break;
          float4 *s0 = reinterpret_cast<float4 *>(xs + q), *s1 = reinterpret_cast<float4 *>(xs + kUpPlane + q);
          float4 *s2 = reinterpret_cast<float4 *>(xs + 2 * kUpPlane + q);
          float4 *s3 = reinterpret_cast<float4 *>(xs + 3 * kUpPlane + q);
          const float4 wh0 = *s0, wl0 = *s1, wh1 = *s2, wl1 = *s3;
          const float a_wh0[4] = {wh0.x, wh0.y, wh0.z, wh0.w}, a_wl0[4] = {wl0.x, wl0.y, wl0.z, wl0.w};
          const float a_wh1[4] = {wh1.x, wh1.y, wh1.z, wh1.w}, a_wl1[4] = {wl1.x, wl1.y, wl1.z, wl1.w};
          const float a_ph0[4] = {ph0[i].x, ph0[i].y, ph0[i].z, ph0[i].w};
          const float a_pl0[4] = {pl0[i].x, pl0[i].y, pl0[i].z, pl0[i].w};
          const float a_ph1[4] = {ph1[i].x, ph1[i].y, ph1[i].z, ph1[i].w};
          const float a_pl1[4] = {pl1[i].x, pl1[i].y, pl1[i].z, pl1[i].w};
          float rh0[4], rl0[4], rh1[4], rl1[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            f2x mh, ml, rh, rl, sh, sl;
            df2_mul(cph, cpl, pk2(a_ph0[k], a_ph1[k]), pk2(a_pl0[k], a_pl1[k]), mh, ml);
            df2_add(mh, ml, pk2(a_wh0[k], a_wh1[k]), pk2(a_wl0[k], a_wl1[k]), rh, rl);
            df2_mul(rh, rl, rh, rl, sh, sl);
            if (d1 == d0) {
              sh &= 0xffffffffull;
              sl &= 0xffffffffull;
            }
            acc2_add(nacc, sh, sl);
            const float2 h2 = upk2(rh), l2 = upk2(rl);
            rh0[k] = h2.x;
            rh1[k] = h2.y;
            rl0[k] = l2.x;
            rl1[k] = l2.y;
          }
          const float4 oh0 = make_float4(rh0[0], rh0[1], rh0[2], rh0[3]);
          const float4 ol0 = make_float4(rl0[0], rl0[1], rl0[2], rl0[3]);
          const float4 oh1 = make_float4(rh1[0], rh1[1], rh1[2], rh1[3]);
          const float4 ol1 = make_float4(rl1[0], rl1[1], rl1[2], rl1[3]);
          *s0 = oh0;
          *s1 = ol0;
          *s2 = oh1;
          *s3 = ol1;
          *reinterpret_cast<float4 *>(x0 + q) = oh0;
          *reinterpret_cast<float4 *>(x0 + ld + q) = ol0;
          if (d1 != d0) {
            *reinterpret_cast<float4 *>(x1 + q) = oh1;
            *reinterpret_cast<float4 *>(x1 + ld + q) = ol1;
          }
        }
      }
      {
        f2x h, l;
        acc2_norm(nacc, h, l);
        double v = df2_lanes_to_f64(h, l);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) wnorm[tid >> 5] += v;
      }
      __syncthreads();
    }
    const uint32_t I0 = F.basis_dn[d0], I1 = F.basis_dn[d1];
    float *__restrict__ z0 = z + d0 * 2 * ld;
    float *__restrict__ z1 = z + d1 * 2 * ld;
    for (int64_t slot = tid; slot < ld; slot += blockDim.x) {
      if (slot >= F.n_up) {                        // padding columns of Z stay zero
        z0[slot] = 0.f;
        z0[ld + slot] = 0.f;
        z1[slot] = 0.f;
        z1[ld + slot] = 0.f;
        continue;
      }
#if HUB_UP_PAIRED
      DfSumP acc{0ull, 0ull, 0ull, {0ull, 0ull}};
#else
      DfSum4 acc{0ull, 0ull, 0ull, {0ull, 0ull, 0ull, 0ull}};
#endif
      const int64_t sl = slot >> 5, lane = slot & 31;
      const uint4 *__restrict__ wa = reinterpret_cast<const uint4 *>(F.sl_add + F.sl_off_add[sl]) + lane;
      const uint4 *__restrict__ wsb = reinterpret_cast<const uint4 *>(F.sl_sub + F.sl_off_sub[sl]) + lane;
      const int na = F.steps_add[sl], ns = F.steps_sub[sl];
      // the (hi d0, hi d1) and (lo d0, lo d1) pairs of staged column C (idle steps read the zero
      // column)
#define HUB_HI(C) pk2(xs[(C)], xs[(C) + 2 * kUpPlane])
#define HUB_LO(C) pk2(xs[(C) + kUpPlane], xs[(C) + 3 * kUpPlane])
#if HUB_UP_PAIRED
      // uint16: one word, both of its scheduled entries as a pair, the low parts to accumulator
      // J (alternating by the word's position in its batch); uint32 (one entry per word): the
      // batch's words x, y as one pair (accumulator 0) and z, w as another (accumulator 1), so
      // that either way an accumulator takes one pair sum per four scheduled entries
#define HUB_WORD(ADD, J, WD)                                                             \
  do {                                                                                   \
    const uint32_t ca_ = (WD) & 0xffffu, cb_ = (WD) >> 16;                               \
    sump_pair(acc, HUB_HI(ca_), HUB_LO(ca_), HUB_HI(cb_), HUB_LO(cb_), (ADD), (J));      \
  } while (0)
#define HUB_J(w) (w)
#else
      // one scheduled entry: J, the low-part accumulator, by the entry's position in its batch
#define HUB_TERM(ADD, J, C)                                                              \
  do {                                                                                   \
    if (ADD)                                                                             \
      sum4_add(acc, HUB_HI(C), HUB_LO(C), (J));                                          \
    else                                                                                 \
      sum4_sub(acc, HUB_HI(C), HUB_LO(C), (J));                                          \
  } while (0)
#define HUB_WORD(ADD, J, WD)                                                             \
  do {                                                                                   \
    if (sizeof(Col) == 2) {                                                              \
      HUB_TERM(ADD, (J), (WD) & 0xffffu);                                                \
      HUB_TERM(ADD, (J) + 1, (WD) >> 16);                                                \
    } else {                                                                             \
      HUB_TERM(ADD, (J), (WD));                                                          \
    }                                                                                    \
  } while (0)
#define HUB_J(w) (((w) * (sizeof(Col) == 2 ? 2 : 1)) & 3)
#endif
      // Full batches of four words run unguarded; the last batch is taken word by word
      // (a word's padding step reads the zero column).  N is uniform over the warp.
#define HUB_GROUP(ADD, W, N)                                                             \
  do {                                                                                   \
    constexpr int kPer = sizeof(Col) == 2 ? 8 : 4;       /* steps per batch */           \
    constexpr int kPerWord = sizeof(Col) == 2 ? 2 : 1;                                   \
    const int nst = (N), nb = (nst + kPer - 1) / kPer;                                   \
    uint4 qn = nb > 0 ? W[0] : make_uint4(0u, 0u, 0u, 0u);                               \
    for (int b = 0; b < nb; ++b) {                                                       \
      const uint4 q = qn;                                                                \
      if (b + 1 < nb) qn = W[(b + 1) * 32];     /* next batch's columns in flight */     \
      const int rem = nst - kPer * b;                                                    \
      if (HUB_UP_PAIRED && sizeof(Col) == 4) {                                           \
        HUB_PAIR32(ADD, 0, q.x, q.y, rem > 1);                                           \
        if (rem > 2) HUB_PAIR32(ADD, 1, q.z, q.w, rem > 3);                              \
      } else {                                                                           \
        HUB_WORD(ADD, HUB_J(0), q.x);                                                    \
        if (rem > kPerWord) HUB_WORD(ADD, HUB_J(1), q.y);                                \
        if (rem > 2 * kPerWord) HUB_WORD(ADD, HUB_J(2), q.z);                            \
        if (rem > 3 * kPerWord) HUB_WORD(ADD, HUB_J(3), q.w);                            \
      }                                                                                  \
    }                                                                                    \
  } while (0)
#if HUB_UP_PAIRED
      // two 32-bit words as one pair, or the first alone when the batch ends after it
#define HUB_PAIR32(ADD, J, WA, WB, BOTH)                                                 \
  do {                                                                                   \
    if (BOTH)                                                                            \
      sump_pair(acc, HUB_HI(WA), HUB_LO(WA), HUB_HI(WB), HUB_LO(WB), (ADD), (J));        \
    else                                                                                 \
      sump_one(acc, HUB_HI(WA), HUB_LO(WA), (ADD), (J));                                 \
  } while (0)
#else
#define HUB_PAIR32(ADD, J, WA, WB, BOTH) \
  do {                                   \
  } while (0)
#endif
      HUB_GROUP(true, wa, na);
      HUB_GROUP(false, wsb, ns);
#undef HUB_GROUP
#undef HUB_PAIR32
#undef HUB_WORD
#undef HUB_J
#undef HUB_TERM
#undef HUB_HI
#undef HUB_LO
      // Z = diag x + t' S for both rows (packed), t' = +-1
      f2x Sh, Sl;
#if HUB_UP_PAIRED
      sump_norm(acc, Sh, Sl);
#else
      sum4_norm(acc, Sh, Sl);
#endif
      if (F.t_neg) {
        Sh ^= kSign2;
        Sl ^= kSign2;
      }
      const uint32_t Iu = F.basis_up_slot[slot];
      const float2 dg0 = utab[__popc(Iu & I0)], dg1 = utab[__popc(Iu & I1)];
      f2x ph, pl, zh, zl;
      df2_mul(pk2(dg0.x, dg1.x), pk2(dg0.y, dg1.y), pk2(xs[slot], xs[slot + 2 * kUpPlane]),
              pk2(xs[slot + kUpPlane], xs[slot + 3 * kUpPlane]), ph, pl);
      df2_add(ph, pl, Sh, Sl, zh, zl);
      const float2 h = upk2(zh), l = upk2(zl);
      z0[slot] = h.x;
      z0[ld + slot] = l.x;
      if (d1 != d0) {
        z1[slot] = h.y;
        z1[ld + slot] = l.y;
      }
    }
    __syncthreads();
  }
  if (kUpd && tid == 0) {                  // wnorm was last written before the loop's final barrier
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += wnorm[k];
    U.partials[blockIdx.x] = t;
  }
}

// ---------------------------------------------------------------------------------------
// Rows too long to stage (e.g. C(18, 9) = 48620 columns, 194 KB per plane): pass 1 runs on
// the transposed matrix instead.  X^T is formed by a tiled transpose, the spin-up hops then
// combine whole rows of X^T exactly as pass 2 combines rows of X (k_dn in mode 2, diagonal
// in the epilogue), and the result is transposed back into Z.  Each transpose moves a
// vector once through HBM; gathers through L2 would instead touch two sectors per term.
// ---------------------------------------------------------------------------------------
constexpr int kTile = 32;

// dst[c][r] = src[r][c] for planar matrices: src has n_r rows (plane length ld_s, n_c valid
// columns), dst has n_c rows of plane length ld_d; dst columns n_r .. ld_d - 1 are zeroed.
// Block (32, 8): a 32 x 32 tile of both planes through shared memory.
__global__ void __launch_bounds__(256) k_transpose(int64_t n_r, int64_t n_c, int64_t ld_s, int64_t ld_d,
                                                   const float *__restrict__ src, float *__restrict__ dst) {
  __shared__ float th[kTile][kTile + 1], tl[kTile][kTile + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t c0 = (int64_t)blockIdx.x * kTile, r0 = (int64_t)blockIdx.y * kTile;
#pragma unroll
  for (int j = 0; j < kTile; j += 8) {
    const int64_t r = r0 + ty + j, c = c0 + tx;
    const bool in = r < n_r && c < n_c;
    th[ty + j][tx] = in ? src[r * 2 * ld_s + c] : 0.f;
    tl[ty + j][tx] = in ? src[r * 2 * ld_s + ld_s + c] : 0.f;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kTile; j += 8) {
    const int64_t c = c0 + ty + j, r = r0 + tx;
    if (c < n_c && r < ld_d) {
      dst[c * 2 * ld_d + r] = th[tx][ty + j];
      dst[c * 2 * ld_d + ld_d + r] = tl[tx][ty + j];
    }
  }
}

// ---------------------------------------------------------------------------------------
// Pass 2: spin-down hops as combinations of whole rows of a column strip, plus the
// epilogue.  Tile = 32 rows x 64 columns; blockIdx.x = row tile (fast), blockIdx.y =
// column strip (slow), so consecutive blocks share a strip.  Lane l of a warp owns the
// columns u0 + 2l, u0 + 2l + 1 (one 64-bit load per plane and row), and sums both with one
// packed FP32x2 TwoSum chain.
// ---------------------------------------------------------------------------------------
#ifndef HUB_DN_LANE_COLS
#define HUB_DN_LANE_COLS 4   // columns per lane in pass 2 (2: 64-bit loads, 4: 128-bit loads)
#endif
constexpr int kDnRows = 32, kDnLaneCols = HUB_DN_LANE_COLS, kDnCols = 32 * kDnLaneCols, kDnThreads = 256;
#ifndef HUB_DN_BATCH
#define HUB_DN_BATCH 2   // strip rows whose loads are issued together in pass 2
#endif
#ifndef HUB_DN_MINB
#define HUB_DN_MINB 5    // resident pass-2 CTAs per SM that the register allocation aims for
#endif

// The hopping side a row-combination pass works on: the rows of the matrix it reads are the
// states of this side, its columns (n_cols valid of ld) the states of the other side.
struct Side {
  int64_t n_rows, n_cols, ld;
  const int32_t *rp, *sp;            // sign-split CSR of this side's hopping matrix
  const void *col;
  int64_t r_begin = 0;               // first row a launch covers (rows r_begin .. n_rows - 1)
};

struct LzArgs {                      // Lanczos epilogue operands
  const float *r_cur;                // r_j   (q_j = r_j / beta_cur)
  const float *r_prev;               // r_{j-1}
  const float2 *coef;                // [0] 1/beta_cur, [1] beta_cur/beta_prev (double-float)
  const double *inv_beta;            // 1/beta_cur (FP64)
  double *partials;                  // alpha partial per block
};

// Coefficients of the recurrence, computed once per step by one thread (keeps FP64
// divisions out of the wide kernels).  scal: [0] alpha_j, [1] beta_cur, [2] beta_prev;
// writes scal[6] = 1/beta_cur and, as double-floats, coef[0] = 1/beta_cur,
// coef[1] = beta_cur/beta_prev (0 at the first step), coef[2] = -alpha_j/beta_cur.
__global__ void k_coeffs(double *__restrict__ scal, float2 *__restrict__ coef) {
  const double a = scal[0], bc = scal[1], bp = scal[2];
  scal[6] = 1.0 / bc;
  coef[0] = f64_to_df(1.0 / bc, 0);
  coef[1] = f64_to_df(bp > 0.0 ? bc / bp : 0.0, 0);
  coef[2] = f64_to_df(-a / bc, 0);
}

// scal[i] = v for the given slots (stream-ordered host -> device scalar writes)
// beta_prev <- beta_cur, beta_cur <- beta_j (scal[2], scal[1], scal[3]) without a host value,
// so that a captured iteration needs no per-iteration arguments.
__global__ void k_rotate_beta(double *__restrict__ scal) {
  const double b_cur = scal[1];
  scal[1] = scal[3];
  scal[2] = b_cur;
}

__global__ void k_set_scal(double *__restrict__ scal, int i0, double v0, int i1, double v1, int i2, double v2) {
  if (i0 >= 0) scal[i0] = v0;
  if (i1 >= 0) scal[i1] = v1;
  if (i2 >= 0) scal[i2] = v2;
}

// Appends (alpha, |r|) = (scal[0], scal[1]) to hist (room for cap pairs) at the count kept
// in scal[7], so that several steps can run between two host read-backs.
__global__ void k_record(double *__restrict__ scal, double *__restrict__ hist, int cap) {
  const int i = (int)scal[7];
  if (i >= 0 && i < cap) {
    hist[2 * i] = scal[0];
    hist[2 * i + 1] = scal[1];
  }
  scal[7] = (double)(i + 1);
}

__device__ __forceinline__ f2x ld2(const float *p) { return *reinterpret_cast<const f2x *>(p); }
__device__ __forceinline__ void st2(float *p, f2x v) { *reinterpret_cast<f2x *>(p) = v; }


// kLane packed pairs per lane: columns u .. u + 2 kLane - 1 (16-byte loads for even kLane)
template <int kLane>
struct Vec {
  f2x v[kLane];
};
template <int kLane>
__device__ __forceinline__ Vec<kLane> ldv(const float *p) {
  Vec<kLane> r;
  if (kLane % 2 == 0) {
#pragma unroll
    for (int i = 0; i < kLane / 2; ++i) {
      const float4 q = reinterpret_cast<const float4 *>(p)[i];
      r.v[2 * i] = pk2(q.x, q.y);
      r.v[(2 * i + 1) % kLane] = pk2(q.z, q.w);
    }
  } else {
    r.v[0] = *reinterpret_cast<const f2x *>(p);
  }
  return r;
}
template <int kLane>
__device__ __forceinline__ void stv(float *p, const Vec<kLane> &a) {
  if (kLane % 2 == 0) {
#pragma unroll
    for (int i = 0; i < kLane / 2; ++i) {
      const float2 x = upk2(a.v[2 * i]), y = upk2(a.v[(2 * i + 1) % kLane]);
      reinterpret_cast<float4 *>(p)[i] = make_float4(x.x, x.y, y.x, y.y);
    }
  } else {
    *reinterpret_cast<f2x *>(p) = a.v[0];
  }
}

// Strip rows k, k + 1 of one sign group (loads issued together) into the lane's accumulators
// as a pair whose low parts go to accumulator J.
template <int kLane, int J, bool kAdd, typename Col>
__device__ __forceinline__ void dn_pair(DfSumP (&acc)[kLane], const Side &S, const char *__restrict__ xh,
                                        const char *__restrict__ xl, int32_t k, uint32_t row_bytes) {
  Vec<kLane> vh[2], vl[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const uint64_t o = (uint64_t)colat<Col>(S.col, k + q) * row_bytes;
    vh[q] = ldv<kLane>(reinterpret_cast<const float *>(xh + o));
    vl[q] = ldv<kLane>(reinterpret_cast<const float *>(xl + o));
  }
#pragma unroll
  for (int i = 0; i < kLane; ++i) sump_pair(acc[i], vh[0].v[i], vl[0].v[i], vh[1].v[i], vl[1].v[i], kAdd, J);
}

// The strip rows ka .. kb - 1 of one sign group (bounds warp-uniform): pairs of rows with
// their low parts into the two accumulators in turn (HUB_DN_BATCH = 4: two pairs' loads in
// flight together), a last single row into accumulator 1.
template <int kLane, bool kAdd, typename Col>
__device__ __forceinline__ void dn_group(DfSumP (&acc)[kLane], const Side &S, const char *__restrict__ xh,
                                         const char *__restrict__ xl, int32_t ka, int32_t kb, uint32_t row_bytes) {
  static_assert(HUB_DN_BATCH == 2 || HUB_DN_BATCH == 4, "HUB_DN_BATCH must be 2 or 4");
  int32_t k = ka;
  for (; k + 4 <= kb; k += 4) {
    if (HUB_DN_BATCH == 4) {
      Vec<kLane> vh[4], vl[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint64_t o = (uint64_t)colat<Col>(S.col, k + q) * row_bytes;
        vh[q] = ldv<kLane>(reinterpret_cast<const float *>(xh + o));
        vl[q] = ldv<kLane>(reinterpret_cast<const float *>(xl + o));
      }
#pragma unroll
      for (int i = 0; i < kLane; ++i) {
        sump_pair(acc[i], vh[0].v[i], vl[0].v[i], vh[1].v[i], vl[1].v[i], kAdd, 0);
        sump_pair(acc[i], vh[2].v[i], vl[2].v[i], vh[3].v[i], vl[3].v[i], kAdd, 1);
      }
    } else {
      dn_pair<kLane, 0, kAdd, Col>(acc, S, xh, xl, k, row_bytes);
      dn_pair<kLane, 1, kAdd, Col>(acc, S, xh, xl, k + 2, row_bytes);
    }
  }
  if (k + 2 <= kb) {
    dn_pair<kLane, 0, kAdd, Col>(acc, S, xh, xl, k, row_bytes);
    k += 2;
  }
  if (k < kb) {
    const uint64_t o = (uint64_t)colat<Col>(S.col, k) * row_bytes;
    const Vec<kLane> vh = ldv<kLane>(reinterpret_cast<const float *>(xh + o));
    const Vec<kLane> vl = ldv<kLane>(reinterpret_cast<const float *>(xl + o));
#pragma unroll
    for (int i = 0; i < kLane; ++i) sump_one(acc[i], vh.v[i], vl.v[i], kAdd, 1);
  }
}

// kMode 0: w (planar double-float, slot order; may alias z) = Z + t S_dn, for hub_apply
//          (the FP64 output in rank order is written afterwards by k_unpermute).
// kMode 1: w = (Z + t S_dn)/beta_cur - (beta_cur/beta_prev) r_prev, partials <- <q_j, w>
//          per block (= <r_j, w>/beta_cur).
// kMode 2: pass 1 on X^T (side = spin up, rows of x are spin-up states, columns spin-down
//          states): w = t S_up + diag x, diag from the two basis strings (no z).
template <typename Col, int kMode>
__global__ void __launch_bounds__(kDnThreads, HUB_DN_MINB) k_dn(const FastView F, const Side S, const float *__restrict__ x,
                                                  const float *z, float *w, LzArgs L) {
  constexpr int kLane = kDnLaneCols / 2;               // packed pairs per lane
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ld = S.ld;
  __shared__ float2 utab[kMode == 2 ? 32 : 1];
  if (kMode == 2) {
    if (threadIdx.x < 32) utab[threadIdx.x] = F.Utab[threadIdx.x];
    __syncthreads();
  }
  const int64_t u = (int64_t)blockIdx.y * kDnCols + kDnLaneCols * lane;
  const int64_t r0 = S.r_begin + (int64_t)blockIdx.x * kDnRows;
  const uint32_t row_bytes = (uint32_t)(2 * ld * sizeof(float));
  DfAcc2 dacc{0ull, 0ull};
  const bool active = u < S.n_cols;                    // u + kDnLaneCols <= ld (see fast_build)
  const char *__restrict__ xh = reinterpret_cast<const char *>(x + u);
  const char *__restrict__ xl = reinterpret_cast<const char *>(x + ld + u);
  for (int rr = warp; rr < kDnRows; rr += kDnThreads / 32) {
    const int64_t d = r0 + rr;
    if (d >= S.n_rows) break;
    const int32_t k0 = S.rp[d], ks = S.sp[d], k1 = S.rp[d + 1];
    float *wr = w + d * 2 * ld;
    if (!active) {
      if (u < ld) {                                      // padding columns of w stay zero
        stv<kLane>(wr + u, Vec<kLane>{});
        stv<kLane>(wr + ld + u, Vec<kLane>{});
      }
      continue;
    }
    DfSumP acc[kLane];
#pragma unroll
    for (int i = 0; i < kLane; ++i) acc[i] = DfSumP{0ull, 0ull, 0ull, {0ull, 0ull}};
    dn_group<kLane, true, Col>(acc, S, xh, xl, k0, ks, row_bytes);
    dn_group<kLane, false, Col>(acc, S, xh, xl, ks, k1, row_bytes);
    Vec<kLane> yh, yl;
    if (kMode == 2) {
      // diag x for the columns (spin-down states) u .. u + kDnLaneCols - 1 of spin-up row d
      const float *xr = x + d * 2 * ld;
      const Vec<kLane> xvh = ldv<kLane>(xr + u), xvl = ldv<kLane>(xr + ld + u);
      const uint32_t Iu = F.basis_up[d];
#pragma unroll
      for (int i = 0; i < kLane; ++i) {
        float2 dg[2];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          const int64_t c = u + 2 * i + b;
          dg[b] = c < S.n_cols ? utab[__popc(Iu & F.basis_dn[c])] : make_float2(0.f, 0.f);
        }
        f2x Sh, Sl, ph, pl;
        sump_norm(acc[i], Sh, Sl);
        if (F.t_neg) {
          Sh ^= kSign2;
          Sl ^= kSign2;
        }
        df2_mul(pk2(dg[0].x, dg[1].x), pk2(dg[0].y, dg[1].y), xvh.v[i], xvl.v[i], ph, pl);
        df2_add(ph, pl, Sh, Sl, yh.v[i], yl.v[i]);
      }
    } else {
      const float *zr = z + d * 2 * ld;
      const Vec<kLane> zh = ldv<kLane>(zr + u), zl = ldv<kLane>(zr + ld + u);
#pragma unroll
      for (int i = 0; i < kLane; ++i) {
        f2x Sh, Sl;
        sump_norm(acc[i], Sh, Sl);
        if (F.t_neg) {
          Sh ^= kSign2;
          Sl ^= kSign2;
        }
        df2_add(zh.v[i], zl.v[i], Sh, Sl, yh.v[i], yl.v[i]);
      }
    }
    if (kMode != 1) {
      stv<kLane>(wr + u, yh);
      stv<kLane>(wr + ld + u, yl);
    } else {
      const float *rc = L.r_cur + d * 2 * ld, *rp = L.r_prev + d * 2 * ld;
      const Vec<kLane> rph = ldv<kLane>(rp + u), rpl = ldv<kLane>(rp + ld + u);
      const Vec<kLane> rch = ldv<kLane>(rc + u), rcl = ldv<kLane>(rc + ld + u);
      // recurrence coefficients, read per row (L1-resident) rather than held across the
      // hopping loop in registers
      const float2 ib = L.coef[0], cp = L.coef[1];
      const f2x ibh = bcast2(ib.x), ibl = bcast2(ib.y), cph = bcast2(cp.x), cpl = bcast2(cp.y);
      Vec<kLane> wh, wl;
#pragma unroll
      for (int i = 0; i < kLane; ++i) {
        f2x ah, al, bh, bl, qh, ql;
        df2_mul(yh.v[i], yl.v[i], ibh, ibl, ah, al);
        df2_mul(cph, cpl, rph.v[i], rpl.v[i], bh, bl);
        df2_sub(ah, al, bh, bl, wh.v[i], wl.v[i]);
        // keep padding columns zero: column u + 2i + 1 (lane b) and u + 2i (both lanes)
        const int64_t c0 = u + 2 * i;
        if (c0 >= S.n_cols) {
          wh.v[i] = 0ull;
          wl.v[i] = 0ull;
        } else if (c0 + 1 >= S.n_cols) {
          wh.v[i] &= 0xffffffffull;
          wl.v[i] &= 0xffffffffull;
        }
        // <r_j, w>, accumulated in double-float, reduced in FP64 and scaled by 1/beta_cur
        df2_mul(rch.v[i], rcl.v[i], wh.v[i], wl.v[i], qh, ql);
        acc2_add(dacc, qh, ql);
      }
      stv<kLane>(wr + u, wh);
      stv<kLane>(wr + ld + u, wl);
    }
  }
  if (kMode == 1) {
    f2x h, l;
    acc2_norm(dacc, h, l);
    double dot = df2_lanes_to_f64(h, l);
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    __shared__ double ws[kDnThreads / 32];
    if (lane == 0) ws[warp] = dot;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int k = 0; k < kDnThreads / 32; ++k) s += ws[k];
      L.partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = s * L.inv_beta[0];
    }
  }
}

// ---------------------------------------------------------------------------------------
// Double-float Lanczos vector kernels (planar rows; padding columns stay zero).  Each
// thread step takes four columns of one row: a 16-byte load per plane, two packed pairs.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void block_sum_to(double v, double *partials) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __shared__ double ws[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) ws[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += ws[k];
    partials[blockIdx.x] = s;
  }
}

// Column quads of a planar vector: quad k of n_rows * (ld / 4) starts at float offset
// row * 2 ld + 4 q (hi) and + ld (lo).  The host keeps n_rows * ld / 4 below 2^32.
struct Quads {
  uint32_t per_row, n;
  int64_t ld;
  __device__ __forceinline__ int64_t at(uint32_t k) const {
    const uint32_t d = k / per_row, q = k - d * per_row;
    return (int64_t)d * 2 * ld + 4 * (int64_t)q;
  }
};
__device__ __forceinline__ void ld4(const float *p, f2x &a, f2x &b) {
  const float4 v = *reinterpret_cast<const float4 *>(p);
  a = pk2(v.x, v.y);
  b = pk2(v.z, v.w);
}
__device__ __forceinline__ void st4(float *p, f2x a, f2x b) {
  const float2 u = upk2(a), v = upk2(b);
  *reinterpret_cast<float4 *>(p) = make_float4(u.x, u.y, v.x, v.y);
}

// r_next = w + coef[2] r_cur = w - (alpha / beta_cur) r_cur  (in place over w);
// partials <- |r_next|^2
__global__ void k_df_update(Quads Q, float *__restrict__ w, const float *__restrict__ r_cur,
                            const float2 *__restrict__ coef, double *__restrict__ partials) {
  const float2 c = coef[2];
  const f2x ch = bcast2(c.x), cl = bcast2(c.y);
  DfAcc2 acc{0ull, 0ull};
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < Q.n; k += (uint64_t)gridDim.x * blockDim.x) {
    const int64_t o = Q.at((uint32_t)k);
    f2x wh[2], wl[2], rh[2], rl[2];
    ld4(w + o, wh[0], wh[1]);
    ld4(w + o + Q.ld, wl[0], wl[1]);
    ld4(r_cur + o, rh[0], rh[1]);
    ld4(r_cur + o + Q.ld, rl[0], rl[1]);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      f2x ph, pl;
      df2_mul(ch, cl, rh[i], rl[i], ph, pl);
      df2_add(ph, pl, wh[i], wl[i], wh[i], wl[i]);
      df2_mul(wh[i], wl[i], wh[i], wl[i], ph, pl);
      acc2_add(acc, ph, pl);
    }
    st4(w + o, wh[0], wh[1]);
    st4(w + o + Q.ld, wl[0], wl[1]);
  }
  f2x h, l;
  acc2_norm(acc, h, l);
  block_sum_to(df2_lanes_to_f64(h, l), partials);
}

// partials <- |v|^2
__global__ void k_df_norm2(Quads Q, const float *__restrict__ v, double *__restrict__ partials) {
  DfAcc2 acc{0ull, 0ull};
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < Q.n; k += (uint64_t)gridDim.x * blockDim.x) {
    const int64_t o = Q.at((uint32_t)k);
    f2x vh[2], vl[2];
    ld4(v + o, vh[0], vh[1]);
    ld4(v + o + Q.ld, vl[0], vl[1]);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      f2x ph, pl;
      df2_mul(vh[i], vl[i], vh[i], vl[i], ph, pl);
      acc2_add(acc, ph, pl);
    }
  }
  f2x h, l;
  acc2_norm(acc, h, l);
  block_sum_to(df2_lanes_to_f64(h, l), partials);
}

// psi += c r, c a double-float coefficient in coef[idx]
__global__ void k_df_axpy(Quads Q, const float2 *__restrict__ coef, int idx, const float *__restrict__ r,
                          float *__restrict__ psi) {
  const float2 a = coef[idx];
  const f2x ah = bcast2(a.x), al = bcast2(a.y);
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < Q.n; k += (uint64_t)gridDim.x * blockDim.x) {
    const int64_t o = Q.at((uint32_t)k);
    f2x ph[2], pl[2], rh[2], rl[2];
    ld4(psi + o, ph[0], ph[1]);
    ld4(psi + o + Q.ld, pl[0], pl[1]);
    ld4(r + o, rh[0], rh[1]);
    ld4(r + o + Q.ld, rl[0], rl[1]);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      f2x mh, ml;
      df2_mul(ah, al, rh[i], rl[i], mh, ml);
      df2_add(mh, ml, ph[i], pl[i], ph[i], pl[i]);
    }
    st4(psi + o, ph[0], ph[1]);
    st4(psi + o + Q.ld, pl[0], pl[1]);
  }
}

// coef[3] = c / scal[1]  (psi coefficient v_j / beta_cur), one thread
__global__ void k_psi_coef(const double *__restrict__ scal, double c, float2 *__restrict__ coef) {
  coef[3] = f64_to_df(c / scal[1], 0);
}

// out (FP64, rank order) = v / |v|  with |v| = scal[idx]; one row per block and step
__global__ void k_df_out_normalised(int64_t n_rows, int64_t n_up, int64_t ld, const float *__restrict__ v,
                                    const double *__restrict__ scal, int idx, const int32_t *__restrict__ slot_of,
                                    double *__restrict__ out) {
  const float2 inv = f64_to_df(1.0 / scal[idx], 0);
  for (int64_t d = blockIdx.x; d < n_rows; d += gridDim.x) {
    const float *__restrict__ row = v + d * 2 * ld;
    for (int64_t u = threadIdx.x; u < n_up; u += blockDim.x) {
      const int32_t s = slot_of[u];
      out[d * n_up + u] = df_to_f64(df_mul(make_float2(row[s], row[ld + s]), inv), 0);
    }
  }
}

// Second-pass recurrence with known coefficients: r_next = (H r_j)/1 ... computed as
// w = (Z + t S)/beta_cur - (beta_cur/beta_prev) r_prev by k_dn<.,1>, then
// r_next = w - (alpha/beta_cur) r_cur by k_df_update (alpha written into scal[0]).

// ---------------------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------------------
static int grid_vec() { return num_sms() * 4; }

struct FastState {
  bool built = false;
  float2 *coef = nullptr;                    // recurrence coefficients (double-float)
  bool col16 = true;
  int32_t *sp[2] = {nullptr, nullptr};
  uint32_t *sl_add = nullptr, *sl_sub = nullptr;
  int32_t *sl_off_add = nullptr, *sl_off_sub = nullptr;
  uint16_t *steps_add = nullptr, *steps_sub = nullptr;
  uint32_t idle_word = 0xffffffffu;
  int32_t *slot_row = nullptr, *slot_of = nullptr;
  uint32_t *basis_slot = nullptr;
  void *col[2] = {nullptr, nullptr};
  float *xdf = nullptr, *zdf = nullptr;      // hub_apply scratch (planar double-float)
  bool staged = true;                        // pass 1 stages rows; else it runs on X^T
  int acc_terms = 0;                         // most terms one low-part accumulator sums (error bound)
  int64_t ld_t = 0;                          // plane length of X^T rows (count_dn padded)
  float *xt = nullptr, *zt = nullptr;        // X^T and Z^T (rows too long to stage)
  float *lz[3] = {nullptr, nullptr, nullptr};
  float *psi = nullptr;
  int *d_range = nullptr;                    // exponent partials [2 G], then scale[4] (k_scale)
  double *d_hist = nullptr, *h_hist = nullptr;  // (alpha, |r|) of the steps since the last read-back
  int *d_err = nullptr;
  int64_t ld = 0;
  // pipelined host-buffer apply: copy stream, per-chunk events, exponent partials, flag
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> events;
  int *d_range_chunks = nullptr, *d_flag = nullptr, *h_flag = nullptr;
  // the multi-vector form: a second copy stream (outputs) and its own events
  cudaStream_t copy_out_stream = nullptr;
  std::vector<cudaEvent_t> many_events;
  // CUDA graphs of one Lanczos iteration (first pass), one per rotation of the three
  // vectors, captured on graph_stream and replayed on the caller's stream; lz_graph_key holds
  // the operands they were captured with
  cudaStream_t graph_stream = nullptr;
  cudaGraphExec_t lz_graph[3] = {nullptr, nullptr, nullptr};
  std::vector<unsigned char> lz_graph_key;
  bool lz_graph_failed = false;
};

static FastState *fast_of(const hub_ctx *h) { return h->fast; }

void fast_release(hub_ctx *h) {
  FastState *f = fast_of(h);
  if (!f) return;
  for (int s = 0; s < 2; ++s) {
    dev_free(f->sp[s]);
    dev_free(f->col[s]);
  }
  dev_free(f->xdf);
  dev_free(f->zdf);
  dev_free(f->xt);
  dev_free(f->zt);
  for (int k = 0; k < 3; ++k) dev_free(f->lz[k]);
  dev_free(f->psi);
  dev_free(f->d_range);
  dev_free(f->d_hist);
  if (f->h_hist) cudaFreeHost(f->h_hist);
  dev_free(f->d_err);
  dev_free(f->d_range_chunks);
  dev_free(f->d_flag);
  if (f->h_flag) cudaFreeHost(f->h_flag);
  for (cudaEvent_t e : f->events) cudaEventDestroy(e);
  if (f->copy_stream) cudaStreamDestroy(f->copy_stream);
  for (cudaEvent_t e : f->many_events) cudaEventDestroy(e);
  if (f->copy_out_stream) cudaStreamDestroy(f->copy_out_stream);
  for (int k = 0; k < 3; ++k)
    if (f->lz_graph[k]) cudaGraphExecDestroy(f->lz_graph[k]);
  if (f->graph_stream) cudaStreamDestroy(f->graph_stream);
  dev_free(f->coef);
  dev_free(f->sl_add);
  dev_free(f->sl_sub);
  dev_free(f->sl_off_add);
  dev_free(f->sl_off_sub);
  dev_free(f->steps_add);
  dev_free(f->steps_sub);
  dev_free(f->slot_row);
  dev_free(f->slot_of);
  dev_free(f->basis_slot);
  delete f;
  h->fast = nullptr;
}

// Plane length of a row: count_up rounded up to a multiple of 4 (16-byte plane starts) and
// of the columns a pass-2 lane loads at once.
static int64_t padded_ld(int64_t n_up) {
  const int64_t a = kDnLaneCols > 4 ? kDnLaneCols : 4;
  return (n_up + a - 1) / a * a;
}

// Parameter magnitudes the double-float window allows (0, or 2^-16 .. 2^16; see kExpSpan).
static bool in_param_range(double v) {
  const double a = std::fabs(v);
  return a == 0.0 || (a >= 0x1p-16 && a <= 0x1p16);
}

// Most terms (pass 2: pair sums) one low-part accumulator of a hopping sum may take: with
// N such additions the product's error is at most max(N + 10.1, 16) u^2 (|H||x|)_n,
// u = 2^-24, so N <= 15 keeps it, with the oracle's own FP64 rounding (2 u^2), below
// 1e-13 (|H||x|)_n = 28.1 u^2.  A row with F_add adding and F_sub subtracting entries gives
// N <= ceil(F_add/4) + ceil(F_sub/4) (9 for the 32-entry rows of the 4x4 lattice).
constexpr int kMaxAccTerms = 15;

// The fast path: uniform t != 0 and U, no site energies (the diagonal is then U k exactly),
// |t| and U / |t| in the parameter range, hopping rows short enough for kMaxAccTerms.
bool fast_eligible(const hub_ctx *h) {
  if (!h->have_hop || !h->have_U || !h->uniform_U || h->has_eps) return false;
  for (double tb : h->t)
    if (tb != h->t[0]) return false;
  if (h->t.empty() || h->t[0] == 0.0 || !in_param_range(h->t[0])) return false;
  if (!in_param_range(h->U0 / std::fabs(h->t[0]))) return false;
  if (h->count[0] <= 0 || h->count[1] <= 0) return false;
  if (h->fast && h->fast->acc_terms > kMaxAccTerms) return false;
  // element quads of a vector are indexed with 32-bit integers
  return h->count[1] * (padded_ld(h->count[0]) / 4) < ((int64_t)1 << 32);
}

// Build the sign-split CSR and double-float tables (called after hub_hopping).
int fast_build(hub_ctx *h) {
  fast_release(h);
  FastState *f = new (std::nothrow) FastState();
  if (!f) return fail(HUB_ERR_OOM, "fast path: host allocation failed");
  h->fast = f;
  f->col16 = h->count[0] <= 65536 && h->count[1] <= 65536;
  f->ld = padded_ld(h->count[0]);
  f->ld_t = padded_ld(h->count[1]);
  f->staged = f->ld + 2 <= kUpPlane;
  const size_t csz = f->col16 ? sizeof(uint16_t) : sizeof(uint32_t);
  for (int s = 0; s < 2; ++s) {
    if (s == 1 && h->shared) break;
    const SpinCSR &c = h->csr[s];
    const int64_t n = h->count[s];
    if (!dev_alloc((void **)&f->sp[s], sizeof(int32_t) * (n + 1), "split CSR") ||
        !dev_alloc(&f->col[s], csz * (size_t)std::max<int64_t>(c.nnz, 1), "split CSR columns"))
      return HUB_ERR_OOM;
    const int g = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 16);
    if (f->col16)
      k_split_csr<uint16_t><<<std::max(g, 1), 256>>>(n, c.rowptr, c.scol, f->sp[s], (uint16_t *)f->col[s]);
    else
      k_split_csr<uint32_t><<<std::max(g, 1), 256>>>(n, c.rowptr, c.scol, f->sp[s], (uint32_t *)f->col[s]);
    HUB_LAUNCH_CHECK();
  }
  // sliced, bank-scheduled H_up for pass 1 (built on the host from the sign-split CSR)
  {
    const int64_t n = h->count[0];
    const int64_t nsl = (n + 31) / 32;
    const int64_t nnz = h->csr[0].nnz;
    std::vector<int32_t> rp(n + 1), spv(n);
    std::vector<uint32_t> col(std::max<int64_t>(nnz, 1));
    HUB_CUDA(cudaMemcpy(rp.data(), h->csr[0].rowptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost));
    HUB_CUDA(cudaMemcpy(spv.data(), f->sp[0], sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    if (f->col16) {
      std::vector<uint16_t> c16(std::max<int64_t>(nnz, 1));
      if (nnz) HUB_CUDA(cudaMemcpy(c16.data(), f->col[0], sizeof(uint16_t) * nnz, cudaMemcpyDeviceToHost));
      for (int64_t k = 0; k < nnz; ++k) col[k] = c16[k];
    } else if (nnz) {
      HUB_CUDA(cudaMemcpy(col.data(), f->col[0], sizeof(uint32_t) * nnz, cudaMemcpyDeviceToHost));
    }
    // slots: rows ordered by (add length, sub length), stable (identity when pass 1 runs
    // on X^T, which has no use for the order)
    std::vector<int32_t> slot_row(n);
    for (int64_t r = 0; r < n; ++r) slot_row[r] = (int32_t)r;
    if (f->staged) std::stable_sort(slot_row.begin(), slot_row.end(), [&](int32_t a, int32_t b) {
      const int la = spv[a] - rp[a], lb = spv[b] - rp[b];
      const int sa = rp[a + 1] - spv[a], sb = rp[b + 1] - spv[b];
      return la != lb ? la > lb : sa > sb;
    });
    std::vector<int32_t> slot_of(n);
    for (int64_t k = 0; k < n; ++k) slot_of[slot_row[k]] = (int32_t)k;
    // terms per low-part accumulator: whole rows of a CSR (pass 2; pass 1 on X^T), or the
    // scheduled steps of a slice (staged pass 1, below)
    auto acc_of_rows = [](const std::vector<int32_t> &r, const std::vector<int32_t> &sp) {
      int m = 0;
      for (size_t k = 0; k + 1 < r.size(); ++k)
        m = std::max(m, (sp[k] - r[k] + 3) / 4 + (r[k + 1] - sp[k] + 3) / 4);
      return m;
    };
    {
      const int sd = h->shared ? 0 : 1;
      std::vector<int32_t> rpd(h->count[sd] + 1), spd(h->count[sd]);
      HUB_CUDA(cudaMemcpy(rpd.data(), h->csr[sd].rowptr, sizeof(int32_t) * rpd.size(), cudaMemcpyDeviceToHost));
      HUB_CUDA(cudaMemcpy(spd.data(), f->sp[sd], sizeof(int32_t) * spd.size(), cudaMemcpyDeviceToHost));
      f->acc_terms = acc_of_rows(rpd, spd);
      if (!f->staged) f->acc_terms = std::max(f->acc_terms, acc_of_rows(rp, spv));
    }
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 16));
    if (!dev_alloc((void **)&f->slot_row, sizeof(int32_t) * n, "slot order") ||
        !dev_alloc((void **)&f->slot_of, sizeof(int32_t) * n, "slot order") ||
        !dev_alloc((void **)&f->basis_slot, sizeof(uint32_t) * n, "basis in slot order"))
      return HUB_ERR_OOM;
    HUB_CUDA(cudaMemcpy(f->slot_row, slot_row.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
    HUB_CUDA(cudaMemcpy(f->slot_of, slot_of.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
    k_to_slots<<<g, 256>>>(n, f->slot_row, h->basis[0], f->basis_slot);
    HUB_LAUNCH_CHECK();
    if (f->staged) {
      // Per slice and group, the lanes' entries are scheduled into steps; the 32-bit loads of
      // one step cost as many shared-memory wavefronts as the most used bank (column mod 32)
      // has distinct columns in it.  Greedy: lanes with the most remaining entries first; each
      // takes a column already used in the step (a broadcast), else one of the most loaded bank
      // that is still under the cap.  Pass 1 is limited by both instruction issue (steps) and
      // shared-memory wavefronts: on the 4x4 lattice a cap of two columns per bank and step
      // runs fastest (steps within a few per cent of the longest lane); a cap of three saves
      // steps but costs 20 % in time, and an adaptive cap (the busiest bank's remaining load
      // over the remaining steps) saves 17 % of the wavefronts for 5 % more steps and runs 1 %
      // slower.
#ifndef HUB_BANK_CAP
#define HUB_BANK_CAP 2   // columns per bank and step: k > 0 fixed, 0 adaptive, -k adaptive capped at k
#endif
      constexpr int kBankCap = HUB_BANK_CAP;
      // idle steps: the zero entry after the staged row when rows are staged, else a sentinel
      const bool staged = f->ld + 2 <= kUpPlane;
      const uint32_t idle = staged ? (uint32_t)f->ld : (f->col16 ? 0xffffu : 0xffffffffu);
      f->idle_word = f->col16 ? (idle | (idle << 16)) : idle;
      const int pack = f->col16 ? 2 : 1;
      std::vector<uint16_t> st[2] = {std::vector<uint16_t>(nsl), std::vector<uint16_t>(nsl)};
      std::vector<int32_t> off[2] = {std::vector<int32_t>(nsl + 1, 0), std::vector<int32_t>(nsl + 1, 0)};
      std::vector<uint32_t> words[2];
      std::vector<std::vector<uint32_t>> warp_steps;  // [S][32] entries of one slice
      for (int64_t sl = 0; sl < nsl; ++sl) {
        for (int grp = 0; grp < 2; ++grp) {
          std::vector<uint32_t> rem[32];
          for (int l = 0; l < 32; ++l) {
            const int64_t slot = sl * 32 + l;
            if (slot >= n) continue;
            const int32_t r = slot_row[slot];
            const int32_t a = grp == 0 ? rp[r] : spv[r], b = grp == 0 ? spv[r] : rp[r + 1];
            for (int32_t k = a; k < b; ++k) rem[l].push_back((uint32_t)slot_of[col[k]]);
          }
          warp_steps.clear();
          std::vector<uint32_t> distinct;
          for (;;) {
            int lanes[32], nl = 0;
            size_t left = 0;
            distinct.clear();
            for (int l = 0; l < 32; ++l)
              if (!rem[l].empty()) {
                lanes[nl++] = l;
                left = std::max(left, rem[l].size());
                distinct.insert(distinct.end(), rem[l].begin(), rem[l].end());
              }
            if (!nl) break;
            std::sort(distinct.begin(), distinct.end());
            distinct.erase(std::unique(distinct.begin(), distinct.end()), distinct.end());
            int bankload[32] = {0};
            for (uint32_t c : distinct) ++bankload[c & 31];
            const int maxload = *std::max_element(bankload, bankload + 32);
            const int need = std::max(1, (int)((maxload + left - 1) / left));
            const int cap = kBankCap > 0 ? kBankCap : (kBankCap < 0 ? std::min(-kBankCap, need) : need);
            std::stable_sort(lanes, lanes + nl, [&](int a, int b) { return rem[a].size() > rem[b].size(); });
            std::vector<uint32_t> step(32, idle);
            uint32_t used_col[32][8];
            int used[32] = {0};
            auto in_step = [&](uint32_t c) {
              const int bk = c & 31;
              for (int i = 0; i < used[bk]; ++i)
                if (used_col[bk][i] == c) return true;
              return false;
            };
            for (int q = 0; q < nl; ++q) {
              const int l = lanes[q];
              int best = -1, best_shared = 0, best_load = 0, best_used = 0;
              for (int e = 0; e < (int)rem[l].size(); ++e) {
                const uint32_t c = rem[l][e];
                const int bk = c & 31;
                const int shared = in_step(c) ? 1 : 0;
                if (!shared && (used[bk] >= cap || used[bk] >= 8)) continue;
                const bool better = best < 0 || shared > best_shared ||
                                    (shared == best_shared && (bankload[bk] > best_load ||
                                                               (bankload[bk] == best_load && used[bk] < best_used)));
                if (better) {
                  best = e;
                  best_shared = shared;
                  best_load = bankload[bk];
                  best_used = used[bk];
                }
              }
              if (best < 0) continue;
              const uint32_t c = rem[l][best];
              step[l] = c;
              if (!best_shared) used_col[c & 31][used[c & 31]++] = c;
              rem[l].erase(rem[l].begin() + best);
            }
            warp_steps.push_back(step);
          }
          const int S = (int)warp_steps.size();
          if (S > 65535) return fail(HUB_ERR_ARG, "fast path: hopping row schedule too long");
          st[grp][sl] = (uint16_t)S;
          if (grp == 1) f->acc_terms = std::max(f->acc_terms, (st[0][sl] + 3) / 4 + (S + 3) / 4);
          const int nw = (S + pack - 1) / pack, nb = (nw + 3) / 4;
          off[grp][sl + 1] = off[grp][sl] + 32 * 4 * nb;
          for (int bt = 0; bt < nb; ++bt)
            for (int l = 0; l < 32; ++l)
              for (int i = 0; i < 4; ++i) {
                const int j = 4 * bt + i;
                uint32_t wd = f->idle_word;
                if (j < nw && pack == 2) {
                  const uint32_t lo = warp_steps[2 * j][l];
                  const uint32_t hi = 2 * j + 1 < S ? warp_steps[2 * j + 1][l] : idle;
                  wd = lo | (hi << 16);
                } else if (j < nw) {
                  wd = warp_steps[j][l];
                }
                words[grp].push_back(wd);
              }
        }
      }
      if (!dev_alloc((void **)&f->sl_off_add, sizeof(int32_t) * (nsl + 1), "slice offsets") ||
          !dev_alloc((void **)&f->sl_off_sub, sizeof(int32_t) * (nsl + 1), "slice offsets") ||
          !dev_alloc((void **)&f->sl_add, sizeof(uint32_t) * std::max<size_t>(words[0].size(), 1), "sliced columns") ||
          !dev_alloc((void **)&f->sl_sub, sizeof(uint32_t) * std::max<size_t>(words[1].size(), 1), "sliced columns") ||
          !dev_alloc((void **)&f->steps_add, sizeof(uint16_t) * nsl, "slice steps") ||
          !dev_alloc((void **)&f->steps_sub, sizeof(uint16_t) * nsl, "slice steps"))
        return HUB_ERR_OOM;
      HUB_CUDA(cudaMemcpy(f->sl_off_add, off[0].data(), sizeof(int32_t) * (nsl + 1), cudaMemcpyHostToDevice));
      HUB_CUDA(cudaMemcpy(f->sl_off_sub, off[1].data(), sizeof(int32_t) * (nsl + 1), cudaMemcpyHostToDevice));
      if (!words[0].empty())
        HUB_CUDA(cudaMemcpy(f->sl_add, words[0].data(), sizeof(uint32_t) * words[0].size(), cudaMemcpyHostToDevice));
      if (!words[1].empty())
        HUB_CUDA(cudaMemcpy(f->sl_sub, words[1].data(), sizeof(uint32_t) * words[1].size(), cudaMemcpyHostToDevice));
      HUB_CUDA(cudaMemcpy(f->steps_add, st[0].data(), sizeof(uint16_t) * nsl, cudaMemcpyHostToDevice));
      HUB_CUDA(cudaMemcpy(f->steps_sub, st[1].data(), sizeof(uint16_t) * nsl, cudaMemcpyHostToDevice));
    }
  }
  if (!dev_alloc((void **)&f->d_err, sizeof(int) * 4, "error flag") ||
      !dev_alloc((void **)&f->coef, sizeof(float2) * 8, "recurrence coefficients"))
    return HUB_ERR_OOM;
  HUB_CUDA(cudaMemset(f->d_err, 0, sizeof(int) * 4));
  HUB_CUDA(cudaDeviceSynchronize());
  f->built = true;
  return HUB_OK;
}

static FastView fast_view(const hub_ctx *h, const FastState *f) {
  FastView v{};
  v.n_up = h->count[0];
  v.n_dn = h->count[1];
  v.ld = f->ld;
  v.basis_up = h->basis[0];
  v.basis_dn = h->basis[1];
  const int sd = h->shared ? 0 : 1;
  v.rp_up = h->csr[0].rowptr;
  v.sp_up = f->sp[0];
  v.rp_dn = h->csr[sd].rowptr;
  v.sp_dn = f->sp[sd];
  v.col_up = f->col[0];
  v.col_dn = f->col[sd];
  v.sl_add = f->sl_add;
  v.sl_sub = f->sl_sub;
  v.sl_off_add = f->sl_off_add;
  v.sl_off_sub = f->sl_off_sub;
  v.steps_add = f->steps_add;
  v.steps_sub = f->steps_sub;
  v.slot_row = f->slot_row;
  v.idle_word = f->idle_word;
  v.basis_up_slot = f->basis_slot;
  // The kernels apply H / |t| (hopping elements -sign(t) esign, exact), the caller's results
  // are scaled by |t| in FP64 (hub_apply) or through alpha, beta (Lanczos).
  const double t = h->t.empty() ? 1.0 : h->t[0];
  v.t_neg = t < 0.0;
  // host double -> double-float: hi = float(a), lo = float(a - hi)
  auto hdf = [](double a) {
    float hi = (float)a;
    return make_float2(hi, (float)(a - (double)hi));
  };
  const double u_scaled = h->U0 / std::fabs(t);
  for (int k = 0; k < 32; ++k) v.Utab[k] = hdf(u_scaled * (double)k);
  v.err = f->d_err;
  v.fail_waits = h->fail_waits ? 1 : 0;
  return v;
}

static Quads quads(const hub_ctx *h, const FastState *f) {
  Quads q;
  q.per_row = (uint32_t)(f->ld / 4);
  q.n = (uint32_t)(h->count[1] * (f->ld / 4));
  q.ld = f->ld;
  return q;
}

static size_t up_smem(const FastState *f) { return sizeof(float) * (3 * (size_t)kUpPlane + (size_t)f->ld + 2); }
constexpr size_t kMaxStage = 224 * 1024;
static_assert(sizeof(float) * 4 * kUpPlane <= kMaxStage, "four staged planes must fit");

// the spin-down side (pass 2 on X) and the spin-up side (pass 1 on X^T)
static Side side_dn(const hub_ctx *h, const FastState *f) {
  const int sd = h->shared ? 0 : 1;
  return Side{h->count[1], h->count[0], f->ld, h->csr[sd].rowptr, f->sp[sd], f->col[sd]};
}
static Side side_up(const hub_ctx *h, const FastState *f) {
  return Side{h->count[0], h->count[1], f->ld_t, h->csr[0].rowptr, f->sp[0], f->col[0]};
}

static dim3 dn_grid(const Side &S) {
  return dim3((unsigned)((S.n_rows - S.r_begin + kDnRows - 1) / kDnRows), (unsigned)((S.n_cols + kDnCols - 1) / kDnCols));
}

template <typename Col, int kMode>
static int launch_dn_t(const FastView &v, const Side &S, const float *x, const float *z, float *w, LzArgs L,
                       cudaStream_t s) {
  const dim3 g = dn_grid(S);
  if (g.y > 65535) return fail(HUB_ERR_ARG, "fast apply: too many column strips");
  k_dn<Col, kMode><<<g, kDnThreads, 0, s>>>(v, S, x, z, w, L);
  HUB_LAUNCH_CHECK();
  return HUB_OK;
}

template <int kMode>
static int launch_dn(const FastState *f, const FastView &v, const Side &S, const float *x, const float *z, float *w,
                     LzArgs L, cudaStream_t s) {
  return f->col16 ? launch_dn_t<uint16_t, kMode>(v, S, x, z, w, L, s)
                  : launch_dn_t<uint32_t, kMode>(v, S, x, z, w, L, s);
}

// dst = src^T for planar matrices (see k_transpose)
static int transpose(int64_t n_r, int64_t n_c, int64_t ld_s, int64_t ld_d, const float *src, float *dst,
                     cudaStream_t s) {
  const dim3 g((unsigned)((n_c + kTile - 1) / kTile), (unsigned)((ld_d + kTile - 1) / kTile));
  if (g.y > 65535) return fail(HUB_ERR_ARG, "fast apply: matrix too large to transpose");
  k_transpose<<<g, dim3(kTile, 8), 0, s>>>(n_r, n_c, ld_s, ld_d, src, dst);
  HUB_LAUNCH_CHECK();
  return HUB_OK;
}

static int ensure_vec(float **p, int64_t n, const char *what);

// z <- pass 1 (x planar double-float); with staged rows, only the row pairs p0 .. p1 - 1
// (p1 < 0: all pairs).  With upd: first x <- x + c r_prev (the Lanczos update, fused into the
// staging of pass 1 when rows are staged, else a separate vector pass), |x|^2 partials into
// upd->partials, their number in *n_part.
static int run_up(hub_ctx *h, FastState *f, float *x, float *z, cudaStream_t s, int64_t p0 = 0, int64_t p1 = -1,
                  const UpdArgs *upd = nullptr, int *n_part = nullptr) {
  const FastView v = fast_view(h, f);
  if (p1 < 0) p1 = (v.n_dn + 1) / 2;
  if ((!f->staged || upd) && (p0 != 0 || p1 != (v.n_dn + 1) / 2))
    return fail(HUB_ERR_STATE, "pass 1: partial range");
  if (p1 <= p0) return HUB_OK;
  int rc;
  const bool fused = upd && f->staged && kFusedUpdate;
  if (upd && !fused) {                 // the update as its own pass, timed on its own
    if ((rc = prof_mark(h, HUB_PROF_UPDATE, true, s))) return rc;
    const int G = grid_vec();
    count_launch(h);
    k_df_update<<<G, 256, 0, s>>>(quads(h, f), x, upd->r_prev, upd->coef, upd->partials);
    HUB_LAUNCH_CHECK();
    if (n_part) *n_part = G;
    if ((rc = prof_mark(h, HUB_PROF_UPDATE, false, s))) return rc;
  }
  if ((rc = prof_mark(h, HUB_PROF_UP, true, s))) return rc;
  if (f->staged) {
    count_launch(h);
    const int threads = v.n_up >= 4096 ? kUpThreads : (v.n_up >= 1024 ? 512 : (v.n_up >= 256 ? 256 : 128));
    const int grid = (int)std::min<int64_t>(p1 - p0, (int64_t)num_sms());
    const size_t smem = up_smem(f);
    const UpdArgs U = fused ? *upd : UpdArgs{};
    if (fused && n_part) *n_part = grid;
#define HUB_UP(C, K)                                                                                      \
  do {                                                                                                    \
    HUB_CUDA(cudaFuncSetAttribute(k_up<C, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxStage)); \
    k_up<C, K><<<grid, threads, smem, s>>>(v, x, z, p0, p1, U);                                          \
  } while (0)
    if (f->col16) {
      if (fused) HUB_UP(uint16_t, true); else HUB_UP(uint16_t, false);
    } else {
      if (fused) HUB_UP(uint32_t, true); else HUB_UP(uint32_t, false);
    }
#undef HUB_UP
    HUB_LAUNCH_CHECK();
  } else {
    const int64_t Dt = h->count[0] * 2 * f->ld_t;
    if ((rc = ensure_vec(&f->xt, Dt, "transposed x")) || (rc = ensure_vec(&f->zt, Dt, "transposed z"))) return rc;
    count_launch(h, 3);
    if ((rc = transpose(h->count[1], h->count[0], f->ld, f->ld_t, x, f->xt, s))) return rc;
    if ((rc = launch_dn<2>(f, v, side_up(h, f), f->xt, nullptr, f->zt, LzArgs{}, s))) return rc;
    if ((rc = transpose(h->count[0], h->count[1], f->ld_t, f->ld, f->zt, z, s))) return rc;
  }
  return prof_mark(h, HUB_PROF_UP, false, s);
}

// pass 2 on the rows r0 .. r1 - 1 of X (r1 < 0: all rows)
static int run_dn(hub_ctx *h, FastState *f, int mode, const float *x, const float *z, float *w, LzArgs L,
                  cudaStream_t s, int64_t r0 = 0, int64_t r1 = -1) {
  const FastView v = fast_view(h, f);
  count_launch(h);
  int rc = prof_mark(h, HUB_PROF_DN, true, s);
  if (rc) return rc;
  Side S = side_dn(h, f);
  S.r_begin = r0;
  if (r1 >= 0) S.n_rows = r1;
  if (S.n_rows <= S.r_begin) return prof_mark(h, HUB_PROF_DN, false, s);
  rc = mode == 0 ? launch_dn<0>(f, v, S, x, z, w, L, s) : launch_dn<1>(f, v, S, x, z, w, L, s);
  if (rc) return rc;
  return prof_mark(h, HUB_PROF_DN, false, s);
}

static int ensure_vec(float **p, int64_t n, const char *what) {
  if (*p) return HUB_OK;
  return dev_alloc((void **)p, sizeof(float) * n, what) ? HUB_OK : HUB_ERR_OOM;
}

static int row_grid(const hub_ctx *h) { return (int)std::min<int64_t>(h->count[1], (int64_t)num_sms() * 8); }

// Exponent partials and scale words of the handle: [2 G] partials, then scale[0..3].
static int *range_buf(FastState *f) {
  if (!f->d_range && !dev_alloc((void **)&f->d_range, sizeof(int) * (2 * grid_vec() + 4), "exponent partials"))
    return nullptr;
  return f->d_range;
}

// hub_apply on the fast path: FP64 in, FP64 out.  A vector outside the double-float window
// (kExpSpan) is multiplied by the FP64 kernel instead: both are launched, the device-side
// flag scale[1] decides which one writes y, so the call stays asynchronous.
int fast_apply_f64(hub_ctx *h, const double *x, double *y, cudaStream_t s) {
  FastState *f = fast_of(h);
  if (!f || !f->built) return fail(HUB_ERR_STATE, "fast apply: not built");
  const int64_t Dp = h->count[1] * 2 * f->ld, D = h->count[0] * h->count[1];
  int rc;
  if ((rc = ensure_vec(&f->xdf, Dp, "apply scratch x")) || (rc = ensure_vec(&f->zdf, Dp, "apply scratch z")))
    return rc;
  const int G = grid_vec();
  int *part = range_buf(f);
  if (!part) return HUB_ERR_OOM;
  int *scale = part + 2 * G;
  count_launch(h, 3);
  k_exp_range<<<G, 256, 0, s>>>(D, x, part);
  k_scale<<<1, 256, 0, s>>>(part, G, scale);
  k_f64_to_df<<<row_grid(h), 256, 0, s>>>(0, h->count[1], h->count[0], f->ld, x, scale, f->slot_row, f->xdf);
  HUB_LAUNCH_CHECK();
  if ((rc = run_up(h, f, f->xdf, f->zdf, s))) return rc;
  if ((rc = run_dn(h, f, 0, f->xdf, f->zdf, f->zdf, LzArgs{}, s))) return rc;
  count_launch(h);
  k_unpermute<<<row_grid(h), 512, 0, s>>>(0, h->count[1], h->count[0], f->ld, f->zdf, f->slot_of, scale,
                                          std::fabs(h->t[0]), y);
  HUB_LAUNCH_CHECK();
  return f64_apply(h, x, y, scale + 1, s);
}

// Row chunks of the host-buffer apply.
constexpr int kHostChunks = 8;

// Row chunk bounds b[0..n] of n_dn rows with relative sizes w (boundaries even, so that no
// pass-1 row pair straddles two chunks; empty chunks dropped); returns n.
static int chunk_bounds(int64_t n_dn, const int (&w)[kHostChunks], int64_t *b) {
  int total = 0;
  for (int c = 0; c < kHostChunks; ++c) total += w[c];
  int n = 0, acc = 0;
  b[0] = 0;
  for (int c = 0; c < kHostChunks; ++c) {
    acc += w[c];
    const int64_t e = c + 1 == kHostChunks ? n_dn : std::min<int64_t>(n_dn, (n_dn * acc / total) & ~(int64_t)1);
    if (e > b[n]) b[++n] = e;
  }
  return n;
}

// Row chunks of a host-buffer apply: the input's last chunk and the output's first chunk are a
// quarter of the others (little pass-1 work is left once the last input chunk has landed, and
// the first output chunk is ready to go back early); per is the largest chunk.
struct HostChunks {
  int64_t bi[kHostChunks + 1], bo[kHostChunks + 1];
  int nci, nco;
  int64_t per;
};

static HostChunks host_chunks(int64_t n_dn) {
  static const int w_in[kHostChunks] = {4, 4, 4, 4, 4, 4, 4, 1}, w_out[kHostChunks] = {1, 4, 4, 4, 4, 4, 4, 4};
  HostChunks C;
  C.nci = chunk_bounds(n_dn, w_in, C.bi);
  C.nco = chunk_bounds(n_dn, w_out, C.bo);
  C.per = 0;
  for (int c = 0; c < C.nci; ++c) C.per = std::max(C.per, C.bi[c + 1] - C.bi[c]);
  for (int c = 0; c < C.nco; ++c) C.per = std::max(C.per, C.bo[c + 1] - C.bo[c]);
  return C;
}

// Scratch of the chunked host-buffer apply: double-float x and z, per-chunk exponent
// partials, the scale words, the route flag (device and pinned host) and the input copy stream.
static int host_pipe_buffers(FastState *f, int64_t Dp) {
  int rc;
  if ((rc = ensure_vec(&f->xdf, Dp, "apply scratch x")) || (rc = ensure_vec(&f->zdf, Dp, "apply scratch z")))
    return rc;
  if (!f->d_range_chunks &&
      !dev_alloc((void **)&f->d_range_chunks, sizeof(int) * 2 * grid_vec() * kHostChunks, "exponent partials"))
    return HUB_ERR_OOM;
  if (!range_buf(f)) return HUB_ERR_OOM;
  if (!f->d_flag && !dev_alloc((void **)&f->d_flag, sizeof(int), "scale flag")) return HUB_ERR_OOM;
  if (!f->h_flag) HUB_CUDA(cudaMallocHost((void **)&f->h_flag, sizeof(int)));
  if (!f->copy_stream) HUB_CUDA(cudaStreamCreateWithFlags(&f->copy_stream, cudaStreamNonBlocking));
  return HUB_OK;
}

static int ensure_events(std::vector<cudaEvent_t> &ev, int n) {
  while ((int)ev.size() < n) {
    cudaEvent_t e;
    HUB_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ev.push_back(e);
  }
  return HUB_OK;
}

// Pass 1 of a host-buffer apply in the input's row chunks (bounds b[0..nc]): each chunk waits
// for its copy (ev_in[c]), then takes its exponent partials (the first chunk also fixes the
// conversion scale), its conversion to double-float and pass 1 on its row pairs.  Ends with
// the whole vector's scale and the route flag, copied to f->h_flag on s (0: converted with the
// right scale; 1: the largest exponent lies outside the first chunk, redo with the global
// scale; 2: outside the double-float window, FP64 kernel).  xd: the FP64 device input.
static int host_pass1(hub_ctx *h, FastState *f, const double *xd, const int64_t *b, int nc, int64_t per,
                      const cudaEvent_t *ev_in, cudaStream_t s) {
  const int64_t n_up = h->count[0];
  const int G = grid_vec();
  int *part = f->d_range_chunks;                 // 2 G exponent partials per chunk
  int *scale = f->d_range + 2 * G;                // [0, 1] first chunk's scale, [2, 3] the whole vector's
  const int rg = (int)std::min<int64_t>(per, (int64_t)num_sms() * 8);
  int rc;
  for (int c = 0; c < nc; ++c) {
    HUB_CUDA(cudaStreamWaitEvent(s, ev_in[c], 0));
    count_launch(h, c == 0 ? 3 : 2);
    k_exp_range<<<G, 256, 0, s>>>((b[c + 1] - b[c]) * n_up, xd + b[c] * n_up, part + 2 * c * G);
    if (c == 0) k_scale<<<1, 256, 0, s>>>(part, G, scale);
    k_f64_to_df<<<rg, 256, 0, s>>>(b[c], b[c + 1], n_up, f->ld, xd, scale, f->slot_row, f->xdf);
    HUB_LAUNCH_CHECK();
    if ((rc = run_up(h, f, f->xdf, f->zdf, s, b[c] / 2, (b[c + 1] + 1) / 2))) return rc;
  }
  count_launch(h);
  k_scale_all<<<1, 256, 0, s>>>(part, G, nc, scale, f->d_flag);
  HUB_LAUNCH_CHECK();
  HUB_CUDA(cudaMemcpyAsync(f->h_flag, f->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  return HUB_OK;
}

// Route flag 1: conversion and pass 1 again, with the whole vector's scale.
static int host_redo(hub_ctx *h, FastState *f, const double *xd, cudaStream_t s) {
  int *scale = f->d_range + 2 * grid_vec();
  count_launch(h);
  k_f64_to_df<<<row_grid(h), 256, 0, s>>>(0, h->count[1], h->count[0], f->ld, xd, scale + 2, f->slot_row, f->xdf);
  HUB_LAUNCH_CHECK();
  return run_up(h, f, f->xdf, f->zdf, s);
}

// Pass 2 in the output's row chunks (bounds b[0..nc]), so that each chunk's result goes back
// while the next is computed (every chunk reads the whole of X by strips; X is read from HBM
// once per chunk): run_dn and the un-permutation into the FP64 device output yd on s, then the
// chunk's copy to y_host on sc (ev_out[c] hands the chunk from s to sc).
static int host_pass2(hub_ctx *h, FastState *f, double *yd, double *y_host, const int64_t *b, int nc, int64_t per,
                      const cudaEvent_t *ev_out, cudaStream_t s, cudaStream_t sc) {
  const int64_t n_up = h->count[0];
  int *scale = f->d_range + 2 * grid_vec();
  const int rg = (int)std::min<int64_t>(per, (int64_t)num_sms() * 8);
  int rc;
  for (int c = 0; c < nc; ++c) {
    if ((rc = run_dn(h, f, 0, f->xdf, f->zdf, f->zdf, LzArgs{}, s, b[c], b[c + 1]))) return rc;
    count_launch(h);
    k_unpermute<<<rg, 512, 0, s>>>(b[c], b[c + 1], n_up, f->ld, f->zdf, f->slot_of, scale + 2,
                                   std::fabs(h->t[0]), yd);
    HUB_LAUNCH_CHECK();
    HUB_CUDA(cudaEventRecord(ev_out[c], s));
    HUB_CUDA(cudaStreamWaitEvent(sc, ev_out[c], 0));
    HUB_CUDA(cudaMemcpyAsync(y_host + b[c] * n_up, yd + b[c] * n_up, sizeof(double) * (b[c + 1] - b[c]) * n_up,
                             cudaMemcpyDeviceToHost, sc));
  }
  return HUB_OK;
}

bool fast_host_pipelined(const hub_ctx *h) {
  const FastState *f = fast_of(h);
  return f && f->built && f->staged && h->count[1] >= 2 * kHostChunks;
}

// The chunked copies and passes of fast_apply_host: input chunks on the copy stream, pass 1
// per chunk, the route flag read on the host, pass 2 and the output chunks back on the copy
// stream.
static int pipeline_host(hub_ctx *h, FastState *f, const double *x_host, double *y_host, double *xd, double *yd,
                         cudaStream_t s, const HostChunks &C) {
  const int64_t n_up = h->count[0], n_dn = h->count[1];
  int rc;
  cudaStream_t sc = f->copy_stream;
  cudaEvent_t *ev_in = f->events.data(), *ev_out = ev_in + kHostChunks, ev_end = ev_in[2 * kHostChunks + 1];
  for (int c = 0; c < C.nci; ++c) {
    HUB_CUDA(cudaMemcpyAsync(xd + C.bi[c] * n_up, x_host + C.bi[c] * n_up,
                             sizeof(double) * (C.bi[c + 1] - C.bi[c]) * n_up, cudaMemcpyHostToDevice, sc));
    HUB_CUDA(cudaEventRecord(ev_in[c], sc));
  }
  if ((rc = host_pass1(h, f, xd, C.bi, C.nci, C.per, ev_in, s))) return rc;
  HUB_CUDA(cudaStreamSynchronize(s));
  if (*f->h_flag == 2) {   // outside the double-float window: the FP64 kernel, one copy back
    if ((rc = f64_apply(h, xd, yd, nullptr, s))) return rc;
    HUB_CUDA(cudaMemcpyAsync(y_host, yd, sizeof(double) * n_dn * n_up, cudaMemcpyDeviceToHost, s));
    HUB_CUDA(cudaStreamSynchronize(s));
    return HUB_OK;
  }
  if (*f->h_flag == 1 && (rc = host_redo(h, f, xd, s))) return rc;
  if ((rc = host_pass2(h, f, yd, y_host, C.bo, C.nco, C.per, ev_out, s, sc))) return rc;
  HUB_CUDA(cudaEventRecord(ev_end, sc));
  HUB_CUDA(cudaStreamWaitEvent(s, ev_end, 0));
  HUB_CUDA(cudaStreamSynchronize(s));
  return HUB_OK;
}

// hub_apply_host on the fast path with staged rows.  The input arrives in row chunks on a copy
// stream while the compute stream converts each chunk and runs pass 1 on its row pairs; after
// pass 2 the output goes back in row chunks while later chunks are un-permuted.  The
// power-of-two scale of the conversion is taken from the first chunk's largest exponent; if
// the whole vector's largest exponent is larger, conversion and pass 1 are redone with it, so
// the result is bit for bit that of hub_apply.  xd, yd: the handle's FP64 device buffers.
int fast_apply_host(hub_ctx *h, const double *x_host, double *y_host, double *xd, double *yd, cudaStream_t s) {
  FastState *f = fast_of(h);
  if (!f || !f->built) return fail(HUB_ERR_STATE, "fast apply: not built");
  const int64_t n_up = h->count[0], n_dn = h->count[1];
  if (!fast_host_pipelined(h)) {   // one piece: copy in, apply, copy out
    HUB_CUDA(cudaMemcpyAsync(xd, x_host, sizeof(double) * n_up * n_dn, cudaMemcpyHostToDevice, s));
    int rc = fast_apply_f64(h, xd, yd, s);
    if (rc) return rc;
    HUB_CUDA(cudaMemcpyAsync(y_host, yd, sizeof(double) * n_up * n_dn, cudaMemcpyDeviceToHost, s));
    HUB_CUDA(cudaStreamSynchronize(s));
    return HUB_OK;
  }
  int rc;
  if ((rc = host_pipe_buffers(f, n_dn * 2 * f->ld))) return rc;
  // events: [kHostChunks] input chunks, [kHostChunks] output chunks, start, end
  if ((rc = ensure_events(f->events, 2 * kHostChunks + 2))) return rc;
  cudaStream_t sc = f->copy_stream;
  const cudaEvent_t ev_start = f->events[2 * kHostChunks];
  const HostChunks C = host_chunks(n_dn);
  HUB_CUDA(cudaEventRecord(ev_start, s));
  HUB_CUDA(cudaStreamWaitEvent(sc, ev_start, 0));
  rc = pipeline_host(h, f, x_host, y_host, xd, yd, s, C);
  if (rc) {   // no copy into or out of the caller's buffers may outlive the call
    cudaStreamSynchronize(sc);
    cudaStreamSynchronize(s);
  }
  return rc;
}


// hub_apply_host_many on the fast path with staged rows.  While the compute stream works on
// vector v, vector v + 1's rows come in on the input copy stream and vector v - 1's output goes
// back on the output copy stream (the host link carries both directions at once).  The FP64
// device buffers alternate between even and odd vectors (xd[v & 1], yd[v & 1]): an input
// buffer is refilled only after the compute stream has finished reading it (x_free), an output
// buffer is rewritten only after its copy to the host has ended (y_free).  Each vector takes
// the same kernels, scale and route as in fast_apply_host, so every result is bit for bit that
// of one hub_apply_host call.  The host waits once per vector, for its route flag after pass 1;
// the next vector's input copies are queued before that wait.
int fast_apply_host_many(hub_ctx *h, int64_t n_vec, const double *x_host, double *y_host, double *const xd[2],
                         double *const yd[2], cudaStream_t s) {
  FastState *f = fast_of(h);
  if (!fast_host_pipelined(h)) return fail(HUB_ERR_STATE, "fast apply: no row-chunk pipeline for this sector");
  const int64_t n_up = h->count[0], n_dn = h->count[1], D = n_up * n_dn;
  int rc;
  if ((rc = host_pipe_buffers(f, n_dn * 2 * f->ld))) return rc;
  if (!f->copy_out_stream) HUB_CUDA(cudaStreamCreateWithFlags(&f->copy_out_stream, cudaStreamNonBlocking));
  // events: [2][kHostChunks] input chunks (by buffer), [kHostChunks] output chunks,
  // x_free[2], y_free[2], start, end
  if ((rc = ensure_events(f->many_events, 3 * kHostChunks + 6))) return rc;
  cudaEvent_t *ev_in = f->many_events.data(), *ev_out = ev_in + 2 * kHostChunks, *x_free = ev_out + kHostChunks,
              *y_free = x_free + 2;
  const cudaEvent_t ev_start = y_free[2], ev_end = y_free[3];
  const HostChunks C = host_chunks(n_dn);
  cudaStream_t si = f->copy_stream, so = f->copy_out_stream;

  auto copy_in = [&](int64_t v) -> int {
    const int p = (int)(v & 1);
    if (v >= 2) HUB_CUDA(cudaStreamWaitEvent(si, x_free[p], 0));
    for (int c = 0; c < C.nci; ++c) {
      HUB_CUDA(cudaMemcpyAsync(xd[p] + C.bi[c] * n_up, x_host + v * D + C.bi[c] * n_up,
                               sizeof(double) * (C.bi[c + 1] - C.bi[c]) * n_up, cudaMemcpyHostToDevice, si));
      HUB_CUDA(cudaEventRecord(ev_in[p * kHostChunks + c], si));
    }
    return HUB_OK;
  };
  auto run = [&]() -> int {
    int rc;
    HUB_CUDA(cudaEventRecord(ev_start, s));
    HUB_CUDA(cudaStreamWaitEvent(si, ev_start, 0));
    HUB_CUDA(cudaStreamWaitEvent(so, ev_start, 0));
    if ((rc = copy_in(0))) return rc;
    for (int64_t v = 0; v < n_vec; ++v) {
      const int p = (int)(v & 1);
      if ((rc = host_pass1(h, f, xd[p], C.bi, C.nci, C.per, ev_in + p * kHostChunks, s))) return rc;
      if (v + 1 < n_vec && (rc = copy_in(v + 1))) return rc;
      HUB_CUDA(cudaStreamSynchronize(s));
      const int route = *f->h_flag;
      if (route == 1 && (rc = host_redo(h, f, xd[p], s))) return rc;
      if (v >= 2) HUB_CUDA(cudaStreamWaitEvent(s, y_free[p], 0));
      if (route == 2) {   // outside the double-float window: the FP64 kernel, one copy back
        if ((rc = f64_apply(h, xd[p], yd[p], nullptr, s))) return rc;
        HUB_CUDA(cudaEventRecord(x_free[p], s));
        HUB_CUDA(cudaEventRecord(ev_out[0], s));
        HUB_CUDA(cudaStreamWaitEvent(so, ev_out[0], 0));
        HUB_CUDA(cudaMemcpyAsync(y_host + v * D, yd[p], sizeof(double) * D, cudaMemcpyDeviceToHost, so));
      } else {
        HUB_CUDA(cudaEventRecord(x_free[p], s));
        if ((rc = host_pass2(h, f, yd[p], y_host + v * D, C.bo, C.nco, C.per, ev_out, s, so))) return rc;
      }
      HUB_CUDA(cudaEventRecord(y_free[p], so));
    }
    HUB_CUDA(cudaEventRecord(ev_end, so));
    HUB_CUDA(cudaStreamWaitEvent(s, ev_end, 0));
    HUB_CUDA(cudaStreamSynchronize(s));
    return HUB_OK;
  };
  rc = run();
  if (rc) {   // no copy into or out of the caller's buffers may outlive the call
    cudaStreamSynchronize(si);
    cudaStreamSynchronize(so);
    cudaStreamSynchronize(s);
  }
  return rc;
}

int fast_check_error(hub_ctx *h) {
  FastState *f = fast_of(h);
  if (!f) return HUB_OK;
  int e = 0;
  HUB_CUDA(cudaMemcpy(&e, f->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    HUB_CUDA(cudaMemset(f->d_err, 0, sizeof(int)));
    return fail(HUB_ERR_TIMEOUT, "a bounded wait for a staged row gave up (row copy never completed)");
  }
  return HUB_OK;
}

// ---------------------------------------------------------------------------------------
// Double-float Lanczos (same recurrence as the FP64 driver; vectors kept unnormalised,
// r_j = beta_{j-1} q_j, so the normalisation is folded into the apply's epilogue).
// scal: [0] alpha_j, [1] beta_cur = |r_j|, [2] beta_prev = |r_{j-1}| (0 at the start),
// [3] beta_j, [5] |psi|, [6] 1/beta_cur.
// ---------------------------------------------------------------------------------------
// Captures `iteration` once per rotation of the three Lanczos vectors (graphs replayed in
// turn on the caller's stream) unless the cached graphs were captured with the same operands.
// Returns false, with the CUDA error state cleared, if capture is not possible; the caller
// then launches each kernel itself.
template <class F>
static bool lz_graphs(hub_ctx *h, FastState *f, float *v0, float *v1, float *v2, F &iteration) {
  if (f->lz_graph_failed) return false;
  std::vector<unsigned char> key;
  auto add = [&](const void *p, size_t n) {
    const unsigned char *b = (const unsigned char *)p;
    key.insert(key.end(), b, b + n);
  };
  const FastView v = fast_view(h, f);
  const Side S = side_dn(h, f);
  const void *ptrs[9] = {v0, v1, v2, f->zdf, h->partials, h->d_scal, h->h_scal, f->coef, f->d_err};
  add(&v, sizeof(v));
  add(&S.n_rows, sizeof(S.n_rows));
  add(&S.ld, sizeof(S.ld));
  add(ptrs, sizeof(ptrs));
  add(&h->partials_n, sizeof(h->partials_n));
  if (f->lz_graph[0] && key == f->lz_graph_key) return true;
  for (int k = 0; k < 3; ++k)
    if (f->lz_graph[k]) {
      cudaGraphExecDestroy(f->lz_graph[k]);
      f->lz_graph[k] = nullptr;
    }
  if (!f->graph_stream && cudaStreamCreateWithFlags(&f->graph_stream, cudaStreamNonBlocking) != cudaSuccess) {
    f->graph_stream = nullptr;
    f->lz_graph_failed = true;
    cudaGetLastError();
    return false;
  }
  float *r[3] = {v0, v1, v2};
  bool ok = true;
  for (int k = 0; k < 3 && ok; ++k) {
    if (cudaStreamBeginCapture(f->graph_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      ok = false;
      break;
    }
    const int rc = iteration(r[k % 3], r[(k + 1) % 3], r[(k + 2) % 3], f->graph_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(f->graph_stream, &g);
    ok = rc == HUB_OK && e == cudaSuccess && g != nullptr &&
         cudaGraphInstantiate(&f->lz_graph[k], g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
  }
  if (!ok) {
    for (int k = 0; k < 3; ++k)
      if (f->lz_graph[k]) {
        cudaGraphExecDestroy(f->lz_graph[k]);
        f->lz_graph[k] = nullptr;
      }
    f->lz_graph_failed = true;
    cudaGetLastError();
    set_error("");
    return false;
  }
  f->lz_graph_key = key;
  return true;
}

int fast_lanczos(hub_ctx *h, const double *x0, int maxit, double tol, double *E0, double *psi_out,
                 int *iters, cudaStream_t s) {
  FastState *f = fast_of(h);
  if (!f || !f->built) return fail(HUB_ERR_STATE, "fast Lanczos: not built");
  const int64_t Dp = h->count[1] * 2 * f->ld;
  int rc;
  for (int k = 0; k < 3; ++k)
    if ((rc = ensure_vec(&f->lz[k], Dp, "Lanczos vector"))) return rc;
  if ((rc = ensure_vec(&f->zdf, Dp, "apply scratch z"))) return rc;
  const int G = grid_vec();
  const Quads Q = quads(h, f);
  const dim3 gd = dn_grid(side_dn(h, f));
  const int64_t n_dn_blocks = (int64_t)gd.x * gd.y;
  constexpr int kTmp = 2048;                      // first-stage slots of the alpha reduction
  if ((rc = ensure_partials(h, std::max<int64_t>(n_dn_blocks, G) + kTmp))) return rc;
  int *part = range_buf(f);
  if (!part) return HUB_ERR_OOM;
  int *scale = part + 2 * G;
  if (!h->d_scal && !dev_alloc((void **)&h->d_scal, sizeof(double) * 8, "Lanczos scalars")) return HUB_ERR_OOM;
  if (!h->h_scal) HUB_CUDA(cudaMallocHost((void **)&h->h_scal, sizeof(double) * 8));
  double *scal = h->d_scal, *P = h->partials;
  float2 *coef = f->coef;

  // r_1 = 2^-shift x0 as double-float (max |r_1| in [1, 2): the FP32 exponent range holds
  // any scale of x0; entries below 2^-126 max |x0| lose bits, which E0 and psi do not
  // notice), scal[1] = |r_1|, scal[0] = scal[2] = 0, coef[2] = 0 (no update before step 1)
  const int64_t D = h->count[0] * h->count[1];
  auto start = [&](float *r) -> int {
    count_launch(h, 6);
    k_exp_range<<<G, 256, 0, s>>>(D, x0, part);
    k_scale<<<1, 256, 0, s>>>(part, G, scale);
    k_f64_to_df<<<row_grid(h), 256, 0, s>>>(0, h->count[1], h->count[0], f->ld, x0, scale, f->slot_row, r);
    k_df_norm2<<<G, 256, 0, s>>>(Q, r, P);
    HUB_LAUNCH_CHECK();
    int rc2 = reduce_partials(P, G, scal + 1, 1, s);
    if (rc2) return rc2;
    k_set_scal<<<1, 1, 0, s>>>(scal, 0, 0.0, 2, 0.0, -1, 0.0);
    k_coeffs<<<1, 1, 0, s>>>(scal, coef);
    HUB_LAUNCH_CHECK();
    return HUB_OK;
  };
  // One step of the recurrence on (rp, wb, ot) = (r_{j-1}, w_{j-1}, free):
  //   pass 1 forms r_j = w_{j-1} - (alpha_{j-1} / |r_{j-1}|) r_{j-1} over wb (fused update),
  //   Z = (H_up + diag) r_j and |r_j|^2;  beta: scal[2] <- |r_{j-1}|, scal[1] <- |r_j|;
  //   pass 2 writes w_j = H r_j / |r_j| - (|r_j| / |r_{j-1}|) r_{j-1} into ot and the alpha
  //   partials <q_j, w_j>;  alpha_j -> scal[0], coef[2] <- -alpha_j / |r_j| for the next
  //   step;  (alpha_j, |r_j|) appended to the step record.  With full == false only pass 1
  //   and the norm (the last step of the second pass).
  auto iteration = [&](float *rp, float *wb, float *ot, cudaStream_t st, bool full) -> int {
    int rc2 = prof_mark(h, HUB_PROF_APPLY, true, st);
    if (rc2) return rc2;
    const UpdArgs U{rp, coef, P};
    int n_norm = 0;
    if ((rc2 = run_up(h, f, wb, f->zdf, st, 0, -1, &U, &n_norm))) return rc2;
    if ((rc2 = reduce_partials(P, n_norm, scal + 3, 1, st))) return rc2;
    count_launch(h, 2);
    k_rotate_beta<<<1, 1, 0, st>>>(scal);
    k_coeffs<<<1, 1, 0, st>>>(scal, coef);
    HUB_LAUNCH_CHECK();
    if (!full) return prof_mark(h, HUB_PROF_APPLY, false, st);
    LzArgs L{wb, rp, coef, scal + 6, P};
    if ((rc2 = run_dn(h, f, 1, wb, f->zdf, ot, L, st))) return rc2;
    if ((rc2 = prof_mark(h, HUB_PROF_APPLY, false, st))) return rc2;
    if ((rc2 = reduce_partials_2stage(P, (int)n_dn_blocks, P + std::max<int64_t>(n_dn_blocks, G), kTmp, scal + 0, 0,
                                      st)))
      return rc2;
    count_launch(h, 2);
    k_coeffs<<<1, 1, 0, st>>>(scal, coef);
    k_record<<<1, 1, 0, st>>>(scal, f->d_hist, kMaxBatchSteps);
    HUB_LAUNCH_CHECK();
    return HUB_OK;
  };
  auto full_step = [&](float *rp, float *wb, float *ot, cudaStream_t st) -> int {
    return iteration(rp, wb, ot, st, true);
  };

  float *rp = f->lz[0], *wb = f->lz[1], *ot = f->lz[2];
  float *const vecs[3] = {f->lz[0], f->lz[1], f->lz[2]};   // step j works on (vecs[j%3], [j+1], [j+2])
  if (!f->d_hist && !dev_alloc((void **)&f->d_hist, sizeof(double) * 2 * kMaxBatchSteps, "step record"))
    return HUB_ERR_OOM;
  if (!f->h_hist) HUB_CUDA(cudaMallocHost((void **)&f->h_hist, sizeof(double) * 2 * kMaxBatchSteps));
  // Replay captured iterations unless profiling (event pairs per launch) is on; rows that
  // take the transposed pass 1 allocate on first use and are not captured.
  const bool graphs = !h->prof && f->staged && lz_graphs(h, f, rp, wb, ot, full_step);
  if ((rc = start(wb))) return rc;
  HUB_CUDA(cudaMemsetAsync(rp, 0, sizeof(float) * Dp, s));
  HUB_CUDA(cudaMemcpyAsync(h->h_scal + 1, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  int shift = 0;
  HUB_CUDA(cudaMemcpyAsync(&shift, scale, sizeof(int), cudaMemcpyDeviceToHost, s));
  HUB_CUDA(cudaStreamSynchronize(s));
  h->start_norm = std::ldexp(h->h_scal[1], shift);   // |x0|
  if (!(h->h_scal[1] > 0.0) || !std::isfinite(h->h_scal[1]))
    return fail(HUB_ERR_ARG, "hub_lanczos_ground: start vector is zero or not finite");

  h->alpha.clear();
  h->beta.clear();
  // the device recurrence runs on H / |t|: its alpha and beta times |t| are those of H
  const double tabs = std::fabs(h->t[0]);
  // Small sectors run several steps per host read-back (a step costs less than the read-back's
  // latency); the steps after the stopping one are discarded, so E0, the iteration count and
  // the coefficients are those of one step per read-back.
  const int batch = D <= kBatchStepsMaxDim ? kMaxBatchSteps : 1;
  double E = 0.0, E_prev = 0.0;
  LowestTracker lowest;
  int status = HUB_ERR_NOCONV;
  int computed = 0;                                // steps run on the device
  bool done = false;
  for (int j = 0; j < maxit && !done;) {
    const int nb = std::min(batch, maxit - j);
    count_launch(h);
    k_set_scal<<<1, 1, 0, s>>>(scal, 7, 0.0, -1, 0.0, -1, 0.0);
    HUB_LAUNCH_CHECK();
    for (int b = 0; b < nb; ++b) {
      const int jj = j + b;
      if (graphs) {
        HUB_CUDA(cudaGraphLaunch(f->lz_graph[jj % 3], s));
      } else if ((rc = full_step(vecs[jj % 3], vecs[(jj + 1) % 3], vecs[(jj + 2) % 3], s))) {
        return rc;
      }
    }
    HUB_CUDA(cudaMemcpyAsync(f->h_hist, f->d_hist, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost, s));
    HUB_CUDA(cudaStreamSynchronize(s));
    computed = j + nb;
    for (int b = 0; b < nb && !done; ++b) {
      const int jj = j + b;
      const double a_dev = f->h_hist[2 * b], r_dev = f->h_hist[2 * b + 1];   // alpha_{jj+1}, |r_{jj+1}|
      if (!std::isfinite(r_dev)) {
        if ((rc = fast_check_error(h))) return rc;       // a given-up wait left the step incomplete
        return fail(HUB_ERR_CUDA, "hub_lanczos_ground: non-finite beta");
      }
      if (jj > 0) {
        // |r_{jj+1}| is beta_jj, the coupling of q_jj and q_{jj+1}: on breakdown T_jj is final
        // and this step's alpha (formed with 1/beta_jj) is dropped
        h->beta.push_back(tabs * r_dev);
        if (tabs * r_dev <= 1e-14 * std::fmax(1.0, std::fabs(h->alpha.back()))) {
          status = HUB_CONVERGED_BREAKDOWN;
          done = true;
          break;
        }
      }
      if (!std::isfinite(a_dev)) {
        if ((rc = fast_check_error(h))) return rc;
        return fail(HUB_ERR_CUDA, "hub_lanczos_ground: non-finite alpha");
      }
      h->alpha.push_back(tabs * a_dev);
      if (tol > 0) E = lowest.next(h->alpha.data(), h->beta.data(), (int)h->alpha.size());   // else at the end
      if (tol > 0 && jj > 0 && std::fabs(E - E_prev) < tol) {
        status = HUB_OK;
        done = true;
        break;
      }
      E_prev = E;
    }
    j += nb;
  }
  if (tol <= 0 && status == HUB_ERR_NOCONV) status = HUB_OK;
  if (tol <= 0 && !h->alpha.empty()) E = tridiag_lowest(h->alpha.data(), h->beta.data(), (int)h->alpha.size());
  if ((rc = fast_check_error(h))) return rc;
  const int last = (int)h->alpha.size() - 1;        // 0-based index of the last kept step
  if (status != HUB_CONVERGED_BREAKDOWN && last >= 0) {
    // beta_k = |w_k - (alpha_k / |r_k|) r_k|: recorded by the following step if it ran in the
    // same batch, else formed now by that step's update (coef[2] is still the last step's)
    if (last + 1 < computed && (last + 1) / batch == last / batch) {
      h->beta.push_back(tabs * f->h_hist[2 * ((last + 1) % batch) + 1]);
    } else {
      count_launch(h);
      k_df_update<<<G, 256, 0, s>>>(Q, vecs[(last + 2) % 3], vecs[(last + 1) % 3], coef, P);
      HUB_LAUNCH_CHECK();
      if ((rc = reduce_partials(P, G, scal + 3, 1, s))) return rc;
      HUB_CUDA(cudaMemcpyAsync(h->h_scal + 3, scal + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
      HUB_CUDA(cudaStreamSynchronize(s));
      h->beta.push_back(tabs * h->h_scal[3]);
    }
  }
  *E0 = E;
  const int k = (int)h->alpha.size();
  if (iters) *iters = k;

  if (psi_out) {
    // second pass, the same deterministic steps again: psi = sum_j v_j q_j = sum_j v_j r_j / |r_j|
    std::vector<double> vv = tridiag_vector(h->alpha.data(), h->beta.data(), k, psi_eigenvalue(h, E));
    if ((rc = ensure_vec(&f->psi, Dp, "ground-state vector"))) return rc;
    rp = f->lz[0];
    wb = f->lz[1];
    ot = f->lz[2];
    if ((rc = start(wb))) return rc;
    HUB_CUDA(cudaMemsetAsync(rp, 0, sizeof(float) * Dp, s));
    HUB_CUDA(cudaMemsetAsync(f->psi, 0, sizeof(float) * Dp, s));
    for (int j = 0; j < k; ++j) {
      if ((rc = iteration(rp, wb, ot, s, j + 1 < k))) return rc;
      count_launch(h, 2);
      k_psi_coef<<<1, 1, 0, s>>>(scal, vv[j], coef);
      k_df_axpy<<<G, 256, 0, s>>>(Q, coef, 3, wb, f->psi);
      HUB_LAUNCH_CHECK();
      float *t0 = rp;
      rp = wb;
      wb = ot;
      ot = t0;
    }
    count_launch(h, 3);
    k_df_norm2<<<G, 256, 0, s>>>(Q, f->psi, P);
    HUB_LAUNCH_CHECK();
    if ((rc = reduce_partials(P, G, scal + 5, 1, s))) return rc;
    k_df_out_normalised<<<row_grid(h), 256, 0, s>>>(h->count[1], h->count[0], f->ld, f->psi, scal, 5, f->slot_of,
                                                    psi_out);
    HUB_LAUNCH_CHECK();
    HUB_CUDA(cudaStreamSynchronize(s));
    if ((rc = fast_check_error(h))) return rc;
  }
  if (status == HUB_ERR_NOCONV) set_error("hub_lanczos_ground: maxit reached before |dE0| < tol");
  return status;
}

}  // namespace hub
