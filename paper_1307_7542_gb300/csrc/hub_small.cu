// hub_small.cu -- the Lanczos ground state of small sectors, one cooperative launch per batch
// of iterations.
//
// Sec. IV's plain Lanczos (the recurrence of hub_lanczos.cu, FP64 throughout) for sectors so
// small that the multi-kernel drivers are bound by launch and synchronisation latency, not by
// the product: the 8-site ring at half filling has 4,900 states and a product of about 45,000
// multiply-adds, while a Lanczos iteration of the multi-kernel drivers is about ten launches
// and a host round trip.  Here one launch runs several iterations and its CTAs meet at a
// barrier between the phases of an iteration: for sectors of at most kSmallClusterMax states
// the launch is one thread-block cluster (k_small_cluster, below: hardware cluster barriers,
// vectors exchanged through distributed shared memory), for larger ones a cooperative grid
// (k_small_lanczos: an arrival counter in global memory, every wait bounded).  In the grid
// form, with the Lanczos vectors kept unnormalised, q_j = c_j S_j (c_0 = 1/|x0|,
// c_j = 1/beta_{j-1}), iteration j is
//   phase 1  w = c_j (H S_j) - beta_{j-1} c_{j-1} S_{j-1};  CTA partials of <q_j, w>
//   barrier  alpha_j = the sum of the partials, in one fixed order in every CTA
//   phase 2  w -= alpha_j q_j, stored as S_{j+1};  CTA partials of |w|^2
//   barrier  beta_j = sqrt(sum); CTA 0 records (alpha_j, beta_j); on breakdown
//            (beta_j <= 1e-14 max(1, |alpha_j|)) every CTA stops.
// The product is Eq. 11 on the count_dn x count_up state matrix (Eq. count2): the diagonal,
// the spin-up hops gathered inside row d and the spin-down hops combining rows, from the CSR
// of a2.  S_j is staged whole in every CTA's shared memory when it fits, so all gathers read
// shared memory; otherwise they read L2 with ld.global.cg (the vectors change between
// barriers and L1 is not coherent across SMs).
//
// E0_j is found on the host, from the recorded coefficients, batch by batch while the next
// batch runs; the stopping rule is the one of the multi-kernel driver on the same alpha_j,
// beta_j, so up to one batch of iterations past the stop is computed and discarded.  The
// ground-state vector is a second launch that repeats the recurrence with the recorded
// coefficients (no reductions: the same operations, so the same vectors) and accumulates
// psi = sum_j y_j q_j, y the eigenvector of T, then normalises psi.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include <cooperative_groups.h>

#include "hub_internal.cuh"

namespace cg = cooperative_groups;

namespace hub {

std::vector<double> tridiag_vector(const double *a, const double *b, int k, double lam);

#ifndef HUB_SMALL_THREADS
#define HUB_SMALL_THREADS 320                  // threads per CTA
#endif
#ifndef HUB_SMALL_PER_THREAD
#define HUB_SMALL_PER_THREAD 1                 // states per thread the grid is sized for
#endif
#ifndef HUB_SMALL_BATCH
#define HUB_SMALL_BATCH 8                      // iterations per launch while E0_j is checked
#endif
constexpr int kSmallThreads = HUB_SMALL_THREADS;
constexpr int kSmallPerThread = HUB_SMALL_PER_THREAD;
constexpr int kSmallBatch = HUB_SMALL_BATCH;
static_assert(kSmallThreads % 32 == 0 && kSmallThreads <= 1024 && kSmallPerThread >= 1 && kSmallBatch >= 1,
              "small-sector launch shape");
constexpr int64_t kSmallStageMax = 25600;      // S_j staged in shared memory up to 200 KB
#ifndef HUB_SMALL_CLUSTER_MAX
#define HUB_SMALL_CLUSTER_MAX 8192             // sectors up to this size run as one CTA cluster (<= 12800)
#endif
constexpr int64_t kSmallClusterMax = HUB_SMALL_CLUSTER_MAX;
constexpr int kSmallClusterCtas = 16;          // CTAs of that cluster at most (non-portable size)
static_assert(kSmallClusterMax >= 0 && 2 * sizeof(double) * kSmallClusterMax <= 200 * 1024,
              "two copies of a cluster-size vector fit in shared memory");
constexpr uint32_t kSmallSpin = 1u << 21;      // polls of a barrier wait before it gives up (about 1 s)

struct SmallState {
  int64_t cap = 0;             // iterations the history holds
  int grid_cap = 0;            // CTAs the partial sums hold
  double *dev = nullptr;       // part [2 grid_cap] | hist [2 cap] | start [1] | coef [cap]
  int *dint = nullptr;         // stat [4] (iterations done, stop flag) | err | pad | arrival counter | pad
  double *host = nullptr;      // pinned: hist [2 cap] | start
  int *hstat = nullptr;        // pinned: stat copies, [2][4] (one per batch in flight)
  cudaEvent_t ev[2] = {nullptr, nullptr};
  bool attr_set = false;
};

struct SmallArgs {
  Ham H;
  int64_t D;
  double *V0, *V1, *V2;        // Lanczos vectors in slot j % 3 (S_j in the grid form, q_j in the cluster form)
  const double *x0;            // start vector (nullptr: SplitMix64 uniform [-1, 1), seed 0)
  double *part, *hist, *start;
  const double *coef;          // mode 1: y
  double *psi;                 // mode 1: output
  int *stat;
  unsigned *bar;
  int *err;
  int j0, j1;                  // iterations j0 .. j1 - 1
  int mode;                    // 0: recurrence with reductions; 1: psi pass
  int fail_waits;              // test hook
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Sum over the CTA's threads in a fixed order; valid in thread 0.
__device__ __forceinline__ double cta_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
  return s;
}

// Synchronisation of all CTAs of one launch, and sums over all its threads in one fixed order
// (the same value in every CTA).  Two forms:
//   cluster: the launch is one thread-block cluster (at most 16 CTAs, one GPC); hardware cluster
//     barriers (about 0.2 us on GB300), each CTA's partial sum read from the others' shared
//     memory;
//   cooperative: all CTAs resident (cooperative launch); an arrival counter in global memory,
//     zeroed before the launch, that only grows (barrier b completes when it reaches (b + 1)
//     times the number of CTAs: one atomic per CTA, about 1.2 us), bounded waits, partial sums
//     in global memory read through L2.
// Partial sums alternate between two slots, so a sum never overwrites the slot a slower CTA may
// still be reading from the previous one.
template <bool kCluster>
struct GridSync {
  unsigned *count;
  int *err;
  double *part;                        // cooperative: [2][G] in global memory
  double *s_part;                      // cluster: [2] in this CTA's shared memory
  int *s_ok;
  double *red, *tot;
  unsigned passed;                     // barriers completed in this launch
  int slot;

  // false: a wait gave up (the error flag is set); the CTA must return
  __device__ bool sync() {
    if constexpr (kCluster) {
      cg::this_cluster().sync();
      return true;
    } else {
      __syncthreads();
      ++passed;
      if (threadIdx.x == 0) {
        const unsigned target = passed * gridDim.x;
        __threadfence();
        int ok = 1;
        if (atomicAdd(count, 1u) + 1u != target) {
          for (uint32_t it = 0; ld_acquire_u32(count) < target; ++it)
            if (it >= kSmallSpin) {
              ok = 0;
              atomicExch(err, 1);
              break;
            }
        }
        __threadfence();
        *s_ok = ok;
      }
      __syncthreads();
      return *s_ok != 0;
    }
  }

  // *out = sum of v over all threads of the launch (every thread gets it)
  __device__ bool total(double v, double *out) {
    v = cta_sum(v, red);
    const int k = slot;
    slot ^= 1;
    const int G = (int)gridDim.x;
    if (kCluster) {
      if (threadIdx.x == 0) s_part[k] = v;
    } else {
      if (threadIdx.x == 0) part[k * G + blockIdx.x] = v;
    }
    if (!sync()) return false;
    if (threadIdx.x < 32) {            // lane r holds the partials of CTAs r, r + 32, ...
      double s = 0.0;
      for (int b = threadIdx.x; b < G; b += 32) {
        if constexpr (kCluster)
          s += *cg::this_cluster().map_shared_rank(s_part + k, (unsigned)b);
        else
          s += __ldcg(part + k * G + b);
      }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (threadIdx.x == 0) *tot = s;
    }
    __syncthreads();
    *out = *tot;
    return true;
  }

  // before a CTA leaves: no other CTA may still read its shared memory
  __device__ void leave() {
    if constexpr (kCluster) cg::this_cluster().sync();
  }
};

// SplitMix64 (seed 0) uniform in [-1, 1) for counter k + 1, as hub_lanczos_ground draws it.
__device__ __forceinline__ double splitmix_uniform(int64_t k) {
  uint64_t z = (uint64_t)(k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

template <bool kStage>
__global__ void __launch_bounds__(kSmallThreads, 1) k_small_lanczos(const SmallArgs A) {
  extern __shared__ double xs[];
  __shared__ double red[kSmallThreads / 32];
  __shared__ double s_tot;
  __shared__ double s_part[2];
  __shared__ double s_diag[kMaxSites + 1];   // uniform U: U * k for k doubly occupied sites
  __shared__ int s_ok;
  GridSync<false> gs{A.bar, A.err, A.part, s_part, &s_ok, red, &s_tot, 0u, 0};
  const Ham &H = A.H;
  const int64_t D = A.D, nu = H.n_up;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  auto V = [&](int k) { return k == 0 ? A.V0 : (k == 1 ? A.V1 : A.V2); };
  if (threadIdx.x <= kMaxSites) s_diag[threadIdx.x] = H.U0 * (double)threadIdx.x;
  __syncthreads();
  // the two exits below come before any access to another CTA's shared memory
  if (A.mode == 0 && __ldcg(A.stat + 1) != 0) return;   // stopped in an earlier launch (all CTAs)
  if (A.fail_waits) {                 // test hook: every CTA takes a given-up wait's exit at once
    if (threadIdx.x == 0) atomicExch(A.err, 1);
    return;
  }
  // scales of S_{j-1} and S_j, and beta_{j-1}.  Within a launch they are carried in registers
  // (every CTA computes the same values): the recorded hist entries are written by CTA 0 after
  // the iteration's last barrier, so other CTAs may not read them back in the same launch.
  double c_prev = 0.0, c, bp = 0.0;
  if (A.j0 == 0) {
    double nn = 0.0;
    for (int64_t n = n0; n < D; n += stride) {
      const double v = A.x0 ? A.x0[n] : splitmix_uniform(n);
      V(0)[n] = v;
      nn = fma(v, v, nn);
    }
    double s2;
    if (!gs.total(nn, &s2)) return;
    const double s = sqrt(s2);
    const bool good = s > 0.0 && isfinite(s);
    if (A.mode == 0 && lead) {
      A.start[0] = s;
      if (!good) A.stat[1] = 2;
    }
    if (!good) {
      gs.leave();
      return;
    }
    c = 1.0 / s;
  } else {                            // the recorded entries of earlier launches
    bp = __ldcg(A.hist + 2 * (A.j0 - 1) + 1);
    c = 1.0 / bp;
    c_prev = 1.0 / (A.j0 >= 2 ? __ldcg(A.hist + 2 * (A.j0 - 2) + 1) : __ldcg(A.start));
  }
  for (int j = A.j0; j < A.j1; ++j) {
    const double *__restrict__ S = V(j % 3);
    const double *__restrict__ Sp = V((j + 2) % 3);
    double *__restrict__ Wv = V((j + 1) % 3);
    if (A.mode == 1) {                // psi += y_j q_j
      const double y = A.coef[j];
      for (int64_t n = n0; n < D; n += stride) {
        const double q = c * __ldcg(S + n);
        A.psi[n] = j == 0 ? y * q : fma(y, q, A.psi[n]);
      }
      if (j + 1 == A.j1) break;
    }
    if (kStage) {
      __syncthreads();                // the previous iteration's reads of xs are done
      for (int64_t k = threadIdx.x; k < D; k += blockDim.x) xs[k] = __ldcg(S + k);
      __syncthreads();
    }
    auto X = [&](int64_t k) -> double { return kStage ? xs[k] : __ldcg(S + k); };
    const double a_rec = A.mode == 1 ? __ldcg(A.hist + 2 * j) : 0.0;
    double dot = 0.0;
    for (int64_t n = n0; n < D; n += stride) {
      const int64_t d = n / nu, u = n - d * nu;
      const double xn = X(n);
      const uint32_t Iu = __ldg(H.basis_up + u), Id = __ldg(H.basis_dn + d);
      const double dg = (H.uniform_U && !H.has_eps) ? s_diag[__popc(Iu & Id)] : diag_of(H, Iu, Id, u, d);
      // spin-up and spin-down hops in two independent chains (the FP64 unit's latency)
      double acc_up = 0.0, acc_dn = 0.0;
      const int64_t row = d * nu;
      for (int32_t k = __ldg(H.rp_up + u), k1 = __ldg(H.rp_up + u + 1); k < k1; ++k)
        acc_up = fma(__ldg(H.val_up + k), X(row + __ldg(H.col_up + k)), acc_up);
      for (int32_t k = __ldg(H.rp_dn + d), k1 = __ldg(H.rp_dn + d + 1); k < k1; ++k)
        acc_dn = fma(__ldg(H.val_dn + k), X((int64_t)__ldg(H.col_dn + k) * nu + u), acc_dn);
      const double acc = fma(dg, xn, acc_up + acc_dn);
      double w = c * acc;
      if (j) w = fma(-bp, c_prev * __ldcg(Sp + n), w);
      const double q = c * xn;
      if (A.mode == 0) {
        Wv[n] = w;
        dot = fma(q, w, dot);
      } else {
        Wv[n] = fma(-a_rec, q, w);
      }
    }
    if (A.mode == 0) {
      double a, b2;
      if (!gs.total(dot, &a)) return;
      double nn = 0.0;
      for (int64_t n = n0; n < D; n += stride) {
        const double w = fma(-a, c * X(n), Wv[n]);
        Wv[n] = w;
        nn = fma(w, w, nn);
      }
      if (!gs.total(nn, &b2)) return;
      const double b = sqrt(b2);
      if (lead) {
        A.hist[2 * j] = a;
        A.hist[2 * j + 1] = b;
        A.stat[0] = j + 1;
      }
      if (b <= 1e-14 * fmax(1.0, fabs(a))) {   // breakdown: the same decision in every CTA
        if (lead) A.stat[1] = 1;
        gs.leave();
        return;
      }
      bp = b;
    } else {                          // psi pass: hist was completed by the earlier launches
      if (!gs.sync()) return;         // S_{j+1} complete before it is read
      bp = __ldcg(A.hist + 2 * j + 1);
    }
    c_prev = c;
    c = 1.0 / bp;
  }
  if (A.mode == 1) {                  // psi /= |psi|
    double nn = 0.0, p2;
    for (int64_t n = n0; n < D; n += stride) {
      const double v = A.psi[n];
      nn = fma(v, v, nn);
    }
    if (!gs.total(nn, &p2)) return;
    const double inv = 1.0 / sqrt(p2);
    for (int64_t n = n0; n < D; n += stride) A.psi[n] *= inv;
  }
  gs.leave();
}

// ---------------------------------------------------------------------------------------
// Sectors of at most kSmallClusterMax states: one thread-block cluster (at most 16 CTAs, one
// GPC).  Here the Lanczos vectors are normalised explicitly (q_j); each thread keeps its states'
// q_j, q_{j-1} and w in registers, and every CTA holds the whole of q_j in shared memory: once
// beta_j is known each CTA writes its slice of q_{j+1} into the shared memory of every CTA of
// the cluster (distributed shared memory), so inside a launch no vector passes through L2.
// Per iteration three cluster barriers: after the <q_j, w> partials, after the |w|^2 partials,
// after the broadcast of q_{j+1} (shared-memory copies alternate, so a broadcast never
// overwrites the copy a slower CTA is still reading).  The last two vectors of a launch also go
// to global memory (slot j % 3), where the next launch of the run finds q_{j0} and q_{j0-1}; the
// psi pass repeats the same operations with the recorded alpha_j, beta_j.
// ---------------------------------------------------------------------------------------
constexpr int kClusterE = 3;        // states per thread at most

__global__ void __launch_bounds__(kSmallThreads, 1) k_small_cluster(const SmallArgs A) {
  extern __shared__ double xs[];      // [2][D]: q_j and q_{j+1}
  __shared__ double red[kSmallThreads / 32];
  __shared__ double s_tot;
  __shared__ double s_part[2];
  __shared__ double s_diag[kMaxSites + 1];
  __shared__ int s_ok;
  GridSync<true> gs{nullptr, nullptr, nullptr, s_part, &s_ok, red, &s_tot, 0u, 0};
  cg::cluster_group cl = cg::this_cluster();
  const Ham &H = A.H;
  const int64_t D = A.D, nu = H.n_up;
  const int G = (int)gridDim.x;
  const int64_t chunk = (D + G - 1) / G;
  const int64_t lo = (int64_t)blockIdx.x * chunk, hi = min(D, lo + chunk);
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  auto V = [&](int k) { return k == 0 ? A.V0 : (k == 1 ? A.V1 : A.V2); };
  if (threadIdx.x <= kMaxSites) s_diag[threadIdx.x] = H.U0 * (double)threadIdx.x;
  __syncthreads();
  // the two exits below come before any access to another CTA's shared memory
  if (A.mode == 0 && __ldcg(A.stat + 1) != 0) return;   // stopped in an earlier launch (all CTAs)
  if (A.fail_waits) {                 // test hook: every CTA takes a given-up wait's exit at once
    if (threadIdx.x == 0) atomicExch(A.err, 1);
    return;
  }
  int64_t nid[kClusterE];
  double q[kClusterE], qp[kClusterE], w[kClusterE], psi[kClusterE];
#pragma unroll
  for (int e = 0; e < kClusterE; ++e) {
    nid[e] = lo + threadIdx.x + (int64_t)e * blockDim.x;
    q[e] = qp[e] = w[e] = psi[e] = 0.0;
  }
  auto own = [&](int e) { return nid[e] < hi; };
  double *cur = xs, *nxt = xs + D;
  // q (q_{j+1}) into every CTA's copy dst and, when `global`, into global slot k: the next launch
  // of the run reads only the last two vectors of this one, so only those are stored (fewer
  // stores for the cluster barrier's release to wait for)
  auto publish = [&](double *dst, int k, bool global) {
#pragma unroll
    for (int e = 0; e < kClusterE; ++e)
      if (own(e)) {
        if (global) V(k)[nid[e]] = q[e];
        for (int r = 0; r < G; ++r) cl.map_shared_rank(dst, (unsigned)r)[nid[e]] = q[e];
      }
  };
  double bp = 0.0;
  if (A.j0 == 0) {                    // q_0 = x0 / |x0|
    double nn = 0.0;
#pragma unroll
    for (int e = 0; e < kClusterE; ++e)
      if (own(e)) {
        q[e] = A.x0 ? A.x0[nid[e]] : splitmix_uniform(nid[e]);
        nn = fma(q[e], q[e], nn);
      }
    double s2;
    gs.total(nn, &s2);
    const double s = sqrt(s2);
    const bool good = s > 0.0 && isfinite(s);
    if (A.mode == 0 && lead) {
      A.start[0] = s;
      if (!good) A.stat[1] = 2;
    }
    if (!good) {
      gs.leave();
      return;
    }
    const double inv = 1.0 / s;
#pragma unroll
    for (int e = 0; e < kClusterE; ++e) q[e] *= inv;
    publish(cur, 0, A.mode == 0);
    cl.sync();
  } else {                            // q_{j0}, q_{j0-1} and beta_{j0-1} from the earlier launches
    bp = __ldcg(A.hist + 2 * (A.j0 - 1) + 1);
    const double *Q = V(A.j0 % 3), *Qp = V((A.j0 + 2) % 3);
#pragma unroll
    for (int e = 0; e < kClusterE; ++e)
      if (own(e)) {
        q[e] = __ldcg(Q + nid[e]);
        qp[e] = __ldcg(Qp + nid[e]);
      }
    for (int64_t k = threadIdx.x; k < D; k += blockDim.x) cur[k] = __ldcg(Q + k);
    __syncthreads();
  }
  for (int j = A.j0; j < A.j1; ++j) {
    if (A.mode == 1) {                // psi += y_j q_j
      const double y = A.coef[j];
#pragma unroll
      for (int e = 0; e < kClusterE; ++e) psi[e] = j == 0 ? y * q[e] : fma(y, q[e], psi[e]);
      if (j + 1 == A.j1) break;
    }
    // w = H q_j - beta_{j-1} q_{j-1}
    double dot = 0.0;
#pragma unroll
    for (int e = 0; e < kClusterE; ++e)
      if (own(e)) {
        const int64_t n = nid[e], d = n / nu, u = n - d * nu;
        const uint32_t Iu = __ldg(H.basis_up + u), Id = __ldg(H.basis_dn + d);
        const double dg = (H.uniform_U && !H.has_eps) ? s_diag[__popc(Iu & Id)] : diag_of(H, Iu, Id, u, d);
        double acc_up = 0.0, acc_dn = 0.0;
        const double *row = cur + d * nu;
        for (int32_t k = __ldg(H.rp_up + u), k1 = __ldg(H.rp_up + u + 1); k < k1; ++k)
          acc_up = fma(__ldg(H.val_up + k), row[__ldg(H.col_up + k)], acc_up);
        for (int32_t k = __ldg(H.rp_dn + d), k1 = __ldg(H.rp_dn + d + 1); k < k1; ++k)
          acc_dn = fma(__ldg(H.val_dn + k), cur[(int64_t)__ldg(H.col_dn + k) * nu + u], acc_dn);
        double v = fma(dg, q[e], acc_up + acc_dn);
        if (j) v = fma(-bp, qp[e], v);
        w[e] = v;
        dot = fma(q[e], v, dot);
      }
    double b;
    if (A.mode == 0) {
      double a, b2;
      gs.total(dot, &a);
      double nn = 0.0;
#pragma unroll
      for (int e = 0; e < kClusterE; ++e)
        if (own(e)) {
          w[e] = fma(-a, q[e], w[e]);
          nn = fma(w[e], w[e], nn);
        }
      gs.total(nn, &b2);
      b = sqrt(b2);
      if (lead) {
        A.hist[2 * j] = a;
        A.hist[2 * j + 1] = b;
        A.stat[0] = j + 1;
      }
      if (b <= 1e-14 * fmax(1.0, fabs(a))) {   // breakdown: the same decision in every CTA
        if (lead) A.stat[1] = 1;
        gs.leave();
        return;
      }
    } else {                          // psi pass: the recorded coefficients
      const double a = __ldcg(A.hist + 2 * j);
#pragma unroll
      for (int e = 0; e < kClusterE; ++e) w[e] = fma(-a, q[e], w[e]);
      b = __ldcg(A.hist + 2 * j + 1);
    }
    const double inv = 1.0 / b;       // q_{j+1} = w / beta_j
#pragma unroll
    for (int e = 0; e < kClusterE; ++e) {
      qp[e] = q[e];
      q[e] = w[e] * inv;
    }
    publish(nxt, (j + 1) % 3, A.mode == 0 && j + 2 >= A.j1);
    cl.sync();
    double *t = cur;
    cur = nxt;
    nxt = t;
    bp = b;
  }
  if (A.mode == 1) {                  // psi /= |psi|
    double nn = 0.0, p2;
#pragma unroll
    for (int e = 0; e < kClusterE; ++e)
      if (own(e)) nn = fma(psi[e], psi[e], nn);
    gs.total(nn, &p2);
    const double inv = 1.0 / sqrt(p2);
#pragma unroll
    for (int e = 0; e < kClusterE; ++e)
      if (own(e)) A.psi[nid[e]] = psi[e] * inv;
  }
  gs.leave();
}

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------

void small_release(hub_ctx *h) {
  SmallState *S = h->small;
  if (!S) return;
  dev_free(S->dev);
  dev_free(S->dint);
  if (S->host) cudaFreeHost(S->host);
  if (S->hstat) cudaFreeHost(S->hstat);
  for (cudaEvent_t e : S->ev)
    if (e) cudaEventDestroy(e);
  delete S;
  h->small = nullptr;
}

bool small_eligible(const hub_ctx *h) {
  return !h->k0 && h->small_max_dim > 0 && h->count[0] * h->count[1] <= h->small_max_dim;
}

int small_check_error(hub_ctx *h) {
  SmallState *S = h->small;
  if (!S || !S->dint) return HUB_OK;
  int e = 0;
  HUB_CUDA(cudaMemcpy(&e, S->dint + 4, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    HUB_CUDA(cudaMemset(S->dint + 4, 0, sizeof(int)));
    return fail(HUB_ERR_TIMEOUT, "a grid barrier of the small-sector Lanczos gave up");
  }
  return HUB_OK;
}

// Launch shape of a small-sector run.
struct SmallShape {
  int grid = 0;
  bool stage = false, cluster = false;
};

static cudaLaunchConfig_t cluster_config(int ctas, size_t smem, cudaStream_t s, cudaLaunchAttribute *attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(kSmallThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr->id = cudaLaunchAttributeClusterDimension;
  attr->val.clusterDim.x = ctas;
  attr->val.clusterDim.y = 1;
  attr->val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Workspace for D states and up to maxit iterations; launch shape.
static int small_setup(hub_ctx *h, int64_t D, int maxit, SmallShape *shape) {
  SmallState *S = h->small;
  if (!S) {
    S = new (std::nothrow) SmallState();
    if (!S) return fail(HUB_ERR_OOM, "small-sector Lanczos: host allocation failed");
    h->small = S;
    for (cudaEvent_t &e : S->ev) HUB_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  const int sms = num_sms();
  const int64_t cap = ((int64_t)std::max(maxit, 64) + 63) / 64 * 64;
  if (cap > S->cap || sms > S->grid_cap) {
    dev_free(S->dev);
    S->dev = nullptr;
    if (S->host) cudaFreeHost(S->host);
    S->host = nullptr;
    S->cap = 0;
    const int64_t nd = 2 * (int64_t)sms + 2 * cap + 1 + cap;
    if (!dev_alloc((void **)&S->dev, sizeof(double) * nd, "small-sector Lanczos scalars")) return HUB_ERR_OOM;
    HUB_CUDA(cudaMallocHost((void **)&S->host, sizeof(double) * (2 * cap + 1)));
    S->cap = cap;
    S->grid_cap = sms;
  }
  if (!S->dint) {
    if (!dev_alloc((void **)&S->dint, sizeof(int) * 8, "small-sector Lanczos flags")) return HUB_ERR_OOM;
    HUB_CUDA(cudaMemset(S->dint, 0, sizeof(int) * 8));
    HUB_CUDA(cudaMallocHost((void **)&S->hstat, sizeof(int) * 8));
  }
  for (int k = 0; k < 3; ++k)
    if (!h->work[k] && !dev_alloc((void **)&h->work[k], sizeof(double) * D, "Lanczos vector")) return HUB_ERR_OOM;
  if (!S->attr_set) {
    HUB_CUDA(cudaFuncSetAttribute(k_small_lanczos<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(double) * kSmallStageMax)));
    HUB_CUDA(cudaFuncSetAttribute(k_small_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(2 * sizeof(double) * kSmallClusterMax)));
    HUB_CUDA(cudaFuncSetAttribute(k_small_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    S->attr_set = true;
  }
  const int64_t per_cta = (int64_t)kSmallThreads * kSmallPerThread;
  const int64_t want = (D + per_cta - 1) / per_cta;
  // one cluster of up to 16 CTAs when the sector is small enough, each CTA's slice holds at most
  // kClusterE states per thread, and such a cluster fits on this GPU
  shape->cluster = false;
  if (D <= kSmallClusterMax) {
    int ctas = (int)std::min<int64_t>(want, kSmallClusterCtas);
    if ((D + ctas - 1) / ctas > (int64_t)kClusterE * kSmallThreads) ctas = kSmallClusterCtas;
    if ((D + ctas - 1) / ctas <= (int64_t)kClusterE * kSmallThreads) {
      cudaLaunchAttribute attr;
      cudaLaunchConfig_t cfg = cluster_config(ctas, 2 * sizeof(double) * (size_t)D, nullptr, &attr);
      int n_clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&n_clusters, k_small_cluster, &cfg) == cudaSuccess && n_clusters >= 1) {
        shape->cluster = true;
        shape->stage = true;
        shape->grid = ctas;
        return HUB_OK;
      }
      (void)cudaGetLastError();      // no such cluster here: the cooperative form
    }
  }
  shape->stage = D <= kSmallStageMax;
  const size_t smem = shape->stage ? sizeof(double) * (size_t)D : 0;
  int per_sm = 0;
  if (shape->stage)
    HUB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_small_lanczos<true>, kSmallThreads, smem));
  else
    HUB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_small_lanczos<false>, kSmallThreads, 0));
  if (per_sm < 1) return fail(HUB_ERR_CUDA, "small-sector Lanczos: kernel cannot be resident");
  shape->grid = (int)std::min<int64_t>(want, std::min<int64_t>(sms, (int64_t)per_sm * sms));
  return HUB_OK;
}

static int small_launch(hub_ctx *h, const SmallArgs &A, const SmallShape &shape, cudaStream_t s) {
  if (shape.cluster) {
    cudaLaunchAttribute attr;
    cudaLaunchConfig_t cfg = cluster_config(shape.grid, 2 * sizeof(double) * (size_t)A.D, s, &attr);
    HUB_CUDA(cudaLaunchKernelEx(&cfg, k_small_cluster, A));
  } else {
    const size_t smem = shape.stage ? sizeof(double) * (size_t)A.D : 0;
    // the arrival counter starts every launch at zero
    HUB_CUDA(cudaMemsetAsync(A.bar, 0, sizeof(unsigned), s));
    void *args[] = {(void *)&A};
    const void *fn = shape.stage ? (const void *)k_small_lanczos<true> : (const void *)k_small_lanczos<false>;
    HUB_CUDA(cudaLaunchCooperativeKernel(fn, dim3(shape.grid), dim3(kSmallThreads), args, smem, s));
  }
  count_launch(h);
  return HUB_OK;
}

int small_lanczos(hub_ctx *h, const double *x0, int maxit, double tol, double *E0, double *psi_out, int *iters,
                  cudaStream_t s) {
  const int64_t D = vec_len(h);
  SmallShape shape;
  int rc = small_setup(h, D, maxit, &shape);
  if (rc) return rc;
  SmallState *S = h->small;
  double *part = S->dev, *hist = part + 2 * S->grid_cap, *start = hist + 2 * S->cap, *coef = start + 1;
  int *stat = S->dint, *err = S->dint + 4;
  unsigned *bar = reinterpret_cast<unsigned *>(S->dint + 6);
  HUB_CUDA(cudaMemsetAsync(stat, 0, sizeof(int) * 4, s));
  HUB_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned) * 2, s));

  SmallArgs A{};
  A.H = h->view();
  A.D = D;
  A.V0 = h->work[0];
  A.V1 = h->work[1];
  A.V2 = h->work[2];
  A.x0 = x0;
  A.part = part;
  A.hist = hist;
  A.start = start;
  A.coef = coef;
  A.psi = psi_out;
  A.stat = stat;
  A.bar = bar;
  A.err = err;
  A.fail_waits = h->fail_waits ? 1 : 0;

  // batches of iterations, two in flight: the host works through one while the next runs
  const int B = tol > 0 ? kSmallBatch : maxit;
  struct Batch {
    int j0, j1, slot;
  } queue[2];
  int head = 0, n_q = 0, next = 0;
  auto enqueue = [&](int slot, int size) -> int {
    const int j0 = next, j1 = std::min(maxit, next + size);
    A.mode = 0;
    A.j0 = j0;
    A.j1 = j1;
    int r = small_launch(h, A, shape, s);
    if (r) return r;
    HUB_CUDA(cudaMemcpyAsync(S->host + 2 * j0, hist + 2 * j0, sizeof(double) * 2 * (j1 - j0),
                             cudaMemcpyDeviceToHost, s));
    if (j0 == 0) HUB_CUDA(cudaMemcpyAsync(S->host + 2 * S->cap, start, sizeof(double), cudaMemcpyDeviceToHost, s));
    HUB_CUDA(cudaMemcpyAsync(S->hstat + 4 * slot, stat, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
    HUB_CUDA(cudaEventRecord(S->ev[slot], s));
    queue[(head + n_q) & 1] = Batch{j0, j1, slot};
    ++n_q;
    next = j1;
    return HUB_OK;
  };
  auto drain = [&]() -> int {
    HUB_CUDA(cudaStreamSynchronize(s));
    return small_check_error(h);
  };

  h->alpha.clear();
  h->beta.clear();
  if ((rc = enqueue(0, B))) return rc;
  if (next < maxit && (rc = enqueue(1, B))) return rc;
  double E = 0.0, E_prev = 0.0, dE_prev = -1.0, dE_last = -1.0;
  LowestTracker lowest;
  int status = HUB_ERR_NOCONV;
  bool stop = false;
  while (n_q > 0 && !stop) {
    const Batch b = queue[head];
    head ^= 1;
    --n_q;
    HUB_CUDA(cudaEventSynchronize(S->ev[b.slot]));
    const int done = S->hstat[4 * b.slot], flag = S->hstat[4 * b.slot + 1];
    if (b.j0 == 0) h->start_norm = S->host[2 * S->cap];
    if (flag == 2) {
      if ((rc = drain())) return rc;
      h->start_norm = S->host[2 * S->cap];
      return fail(HUB_ERR_ARG, "hub_lanczos_ground: start vector is zero or not finite");
    }
    if (done < b.j1 && flag == 0) {   // the launch stopped without a breakdown: a barrier gave up
      if ((rc = drain())) return rc;
      return fail(HUB_ERR_CUDA, "hub_lanczos_ground: small-sector launch stopped early");
    }
    const int last = std::min(done, b.j1);
    for (int j = b.j0; j < last; ++j) {
      const double a = S->host[2 * j], bb = S->host[2 * j + 1];
      if (!std::isfinite(a) || !std::isfinite(bb)) {
        if ((rc = drain())) return rc;
        return fail(HUB_ERR_CUDA, "hub_lanczos_ground: non-finite alpha/beta");
      }
      h->alpha.push_back(a);
      h->beta.push_back(bb);
      if (tol > 0) E = lowest.next(h->alpha.data(), h->beta.data(), (int)h->alpha.size());   // else at the end
      if (tol > 0 && j > 0 && std::fabs(E - E_prev) < tol) {
        status = HUB_OK;
        stop = true;
        break;
      }
      if (tol > 0 && j > 0) {
        dE_prev = dE_last;
        dE_last = std::fabs(E - E_prev);
      }
      E_prev = E;
      if (bb <= 1e-14 * std::fmax(1.0, std::fabs(a))) {
        status = HUB_CONVERGED_BREAKDOWN;
        stop = true;
        break;
      }
    }
    if (!stop && flag == 1) {         // the device stopped on a breakdown the host did not see
      status = HUB_CONVERGED_BREAKDOWN;
      stop = true;
    }
    if (!stop && next < maxit) {
      // Batch size: once |dE0| falls geometrically, the iterations still needed are about
      // log(tol / dE) / log(rate); a batch that would run past the predicted stop is cut
      // short, and none is started while the one in flight is predicted to reach it (the
      // stopping rule itself is unchanged: the predictions only move launch boundaries)
      int size = B;
      bool wait = false;
      if (tol > 0 && dE_prev > 0.0 && dE_last > 0.0 && dE_last < 0.95 * dE_prev) {
        const double need = std::log(tol / dE_last) / std::log(dE_last / dE_prev);
        const int ahead = next - (int)h->alpha.size();    // launched, not yet seen
        const int more = (int)std::ceil(need) - ahead;
        if (more <= 0 && n_q > 0)
          wait = true;
        else
          size = std::max(1, std::min(B, more + 1));
      }
      if (!wait && (rc = enqueue(b.slot, size))) return rc;
    }
  }
  if ((rc = drain())) return rc;
  if (tol <= 0 && status == HUB_ERR_NOCONV) status = HUB_OK;
  if (tol <= 0 && !h->alpha.empty()) E = tridiag_lowest(h->alpha.data(), h->beta.data(), (int)h->alpha.size());
  *E0 = E;
  const int k = (int)h->alpha.size();
  if (iters) *iters = k;

  if (psi_out && k > 0) {
    const std::vector<double> y = tridiag_vector(h->alpha.data(), h->beta.data(), k, psi_eigenvalue(h, E));
    std::copy(y.begin(), y.end(), S->host);
    HUB_CUDA(cudaMemcpyAsync(coef, S->host, sizeof(double) * k, cudaMemcpyHostToDevice, s));
    // the history on the device still holds alpha_j, beta_j for j < k (later batches only
    // wrote higher j)
    A.mode = 1;
    A.j0 = 0;
    A.j1 = k;
    if ((rc = small_launch(h, A, shape, s))) return rc;
    if ((rc = drain())) return rc;
  }
  if (status == HUB_ERR_NOCONV) set_error("hub_lanczos_ground: maxit reached before |dE0| < tol");
  return status;
}

}  // namespace hub

using namespace hub;

extern "C" int hub_set_small_dim(hub_t h, int64_t max_dim) {
  if (!h || max_dim < 0) return fail(HUB_ERR_ARG, "hub_set_small_dim: bad argument");
  h->small_max_dim = max_dim;
  return HUB_OK;
}
