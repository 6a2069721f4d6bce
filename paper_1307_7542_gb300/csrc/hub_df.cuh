// hub_df.cuh -- double-float arithmetic on the FP32 pipe, and FP64 <-> double-float
// conversions done with integer instructions.
//
// On this GPU the FP64 unit issues about 0.5e12 instructions/s (conversions between
// FP32 and FP64 run there too), against about 36e12/s for FP32 and integer work.  The
// fast apply therefore keeps vectors as pairs (hi, lo) of FP32 numbers with
// x ~= hi + lo (about 48 significant bits) and sums with the error-free transformation
// TwoSum (Knuth, TAOCP vol. 2, 4.2.2; Moller 1965): s = a + b, e = (a - (s - bb)) +
// (b - bb) with bb = s - a gives a + b = s + e exactly.  Products use the FMA-based
// TwoProd (p = a*b, e = fma(a, b, -p) is exact).  Nothing here uses an FP64 instruction
// except the single add in df_to_f64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hub {

// (s, e) with s + e == a + b exactly (round-to-nearest FP32, no overflow).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (s, e) with s + e == a + b exactly, valid when |a| >= |b| (or a == 0).
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// Accumulator: the exact sum of the high parts is kept as H plus the rounding errors,
// which go to L together with the low parts (used for the long dot products of Lanczos;
// the hopping sums of the product use the compensated DfSumP or DfSum4 below).
struct DfAcc {
  float H, L;
};

__device__ __forceinline__ void acc_add(DfAcc &a, float2 v) {
  float s, e;
  two_sum(a.H, v.x, s, e);
  a.H = s;
  a.L = __fadd_rn(__fadd_rn(a.L, v.y), e);
}

__device__ __forceinline__ void acc_sub(DfAcc &a, float2 v) {
  float s, e;
  two_sum(a.H, -v.x, s, e);
  a.H = s;
  a.L = __fadd_rn(__fsub_rn(a.L, v.y), e);
}

// Normalised double-float value of an accumulator.
__device__ __forceinline__ float2 acc_value(const DfAcc &a) {
  float s, e;
  two_sum(a.H, a.L, s, e);
  return make_float2(s, e);
}

// a + b for normalised double-floats (sloppy addition: TwoSum of the high parts).
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  float s, e;
  two_sum(a.x, b.x, s, e);
  e = __fadd_rn(e, __fadd_rn(a.y, b.y));
  float r, f;
  fast_two_sum(s, e, r, f);
  return make_float2(r, f);
}

// a * b for double-floats (TwoProd of the high parts plus the cross terms).
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  float r, f;
  fast_two_sum(p, e, r, f);
  return make_float2(r, f);
}

// a * b + c for double-floats.
__device__ __forceinline__ float2 df_fma(float2 a, float2 b, float2 c) { return df_add(df_mul(a, b), c); }

// ---------------------------------------------------------------------------------------
// Two independent double-float accumulators advanced together with the packed FP32x2
// instructions of sm_100+ (add.rn.f32x2 / sub.rn.f32x2: two IEEE round-to-nearest FP32
// operations per instruction), so TwoSum costs 6 instructions for two sums.
// ---------------------------------------------------------------------------------------
typedef unsigned long long f2x;   // (lane a, lane b) packed in one 64-bit register

__device__ __forceinline__ f2x pk2(float a, float b) {
  f2x r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 upk2(f2x r) {
  float a, b;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
  return make_float2(a, b);
}
// HUB_F32X2 0 issues two scalar round-to-nearest FP32 operations instead of one packed
// instruction: the same results bit for bit (each lane is one IEEE add either way).
#ifndef HUB_F32X2
#define HUB_F32X2 1
#endif
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
#if HUB_F32X2
  f2x r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
#else
  const float2 u = upk2(a), v = upk2(b);
  return pk2(__fadd_rn(u.x, v.x), __fadd_rn(u.y, v.y));
#endif
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
#if HUB_F32X2
  f2x r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
#else
  const float2 u = upk2(a), v = upk2(b);
  return pk2(__fsub_rn(u.x, v.x), __fsub_rn(u.y, v.y));
#endif
}

__device__ __forceinline__ f2x bcast2(float a) { return pk2(a, a); }

// sign bits of both lanes (XOR negates both exactly)
constexpr f2x kSign2 = 0x8000000080000000ull;

struct DfAcc2 {
  f2x H, L;   // high parts (exact running sums) and low parts + TwoSum errors, per lane
};

// a += v (v = vh + vl per lane): TwoSum of the high parts, errors and low parts into L.
__device__ __forceinline__ void acc2_add(DfAcc2 &a, f2x vh, f2x vl) {
  const f2x s = add2(a.H, vh);
  const f2x bb = sub2(s, a.H);
  const f2x e = add2(sub2(a.H, sub2(s, bb)), sub2(vh, bb));
  a.H = s;
  a.L = add2(add2(a.L, vl), e);
}

// a -= v: the TwoSum of (a.H, -vh) written with subtractions (negation is exact, so this
// is the same error-free transformation as acc2_add of -v).
__device__ __forceinline__ void acc2_sub(DfAcc2 &a, f2x vh, f2x vl) {
  const f2x s = sub2(a.H, vh);
  const f2x bb = sub2(s, a.H);
  const f2x e = sub2(sub2(a.H, sub2(s, bb)), add2(vh, bb));
  a.H = s;
  a.L = add2(sub2(a.L, vl), e);
}

// ---------------------------------------------------------------------------------------
// Compensated paired sum for the hopping terms of the product (sums of +-v, v = vh + vl a
// normalised double-float, |vl| <= u |vh|, u = 2^-24).  Per term:
//   (H, e) = TwoSum(H, vh)     H: the FP32 running sum of the high parts, e its exact error
//   (L, f) = TwoSum(L, e)      the errors summed exactly as well ...
//   C += f                     ... up to the plain sum of their own errors
//   V[j] += vl                 low parts, plainly, in four accumulators used in turn
// so that H + L + C_exact + sum_j V_j_exact is the exact sum.  Error over F terms (A =
// sum |v|): each e is at most u A, so |L| <= F u A and |f| <= F u^2 A, and C's roundings
// add at most F^3 u^3 A / 2 (1e-3 u^2 A for F = 32); accumulator V[j] adds n_j - 1
// roundings of at most u sum |vl| over its n_j terms, i.e. at most (max_j n_j - 1) u^2 A.
// The closing steps (V into L by TwoSum, then H + L + C) round once more, by at most
// u^2 |H + L| + u |C|.  The plain form (e and vl summed in one FP32 word) can reach
// F^2 u^2 A, far above the product's tolerance (1e-13 A ~ 28 u^2 A); this one costs 14
// packed instructions per term against 8.
// ---------------------------------------------------------------------------------------
struct DfSum4 {
  f2x H, L, C, V[4];
};

// (s, err) = TwoSum(a, b) per lane
__device__ __forceinline__ void two_sum2(f2x a, f2x b, f2x &s, f2x &err) {
  s = add2(a, b);
  const f2x bb = sub2(s, a);
  err = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
// (s, err) = TwoSum(a, -b) per lane, written with subtractions
__device__ __forceinline__ void two_diff2(f2x a, f2x b, f2x &s, f2x &err) {
  s = sub2(a, b);
  const f2x bb = sub2(s, a);
  err = sub2(sub2(a, sub2(s, bb)), add2(b, bb));
}

// a += v, low part into V[j] (j a compile-time constant after unrolling, so that V stays
// in registers)
__device__ __forceinline__ void sum4_add(DfSum4 &a, f2x vh, f2x vl, int j) {
  f2x e, f;
  two_sum2(a.H, vh, a.H, e);
  two_sum2(a.L, e, a.L, f);
  a.C = add2(a.C, f);
  a.V[j & 3] = add2(a.V[j & 3], vl);
}
// a -= v (negation is exact: the same steps on -v)
__device__ __forceinline__ void sum4_sub(DfSum4 &a, f2x vh, f2x vl, int j) {
  f2x e, f;
  two_diff2(a.H, vh, a.H, e);
  two_sum2(a.L, e, a.L, f);
  a.C = add2(a.C, f);
  a.V[j & 3] = sub2(a.V[j & 3], vl);
}
// Normalised (hi, lo) per lane of the sum.
__device__ __forceinline__ void sum4_norm(const DfSum4 &a, f2x &h, f2x &l) {
  f2x L = a.L, C = a.C, f;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    two_sum2(L, a.V[j], L, f);
    C = add2(C, f);
  }
  f2x s, e;
  two_sum2(a.H, L, s, e);
  two_sum2(s, add2(e, C), h, l);
}

// The same sum with the low parts of two terms added together first (one rounding of at
// most u |vl_a + vl_b|) and the pair sums going to two accumulators in turn: per pair the
// same instruction count as DfSum4, three registers pairs fewer.  A row of F_add + F_sub
// terms puts at most ceil(F_add/4) + ceil(F_sub/4) pair sums (or single last terms) into
// one accumulator.
struct DfSumP {
  f2x H, L, C, V[2];
};

__device__ __forceinline__ void sump_hi(DfSumP &a, f2x vh, bool add) {
  f2x e, f;
  if (add)
    two_sum2(a.H, vh, a.H, e);
  else
    two_diff2(a.H, vh, a.H, e);
  two_sum2(a.L, e, a.L, f);
  a.C = add2(a.C, f);
}
// a += va + vb (add) or a -= va + vb, the pair's low parts into V[j]
__device__ __forceinline__ void sump_pair(DfSumP &a, f2x vha, f2x vla, f2x vhb, f2x vlb, bool add, int j) {
  sump_hi(a, vha, add);
  sump_hi(a, vhb, add);
  const f2x v = add2(vla, vlb);
  a.V[j & 1] = add ? add2(a.V[j & 1], v) : sub2(a.V[j & 1], v);
}
__device__ __forceinline__ void sump_one(DfSumP &a, f2x vh, f2x vl, bool add, int j) {
  sump_hi(a, vh, add);
  a.V[j & 1] = add ? add2(a.V[j & 1], vl) : sub2(a.V[j & 1], vl);
}
__device__ __forceinline__ void sump_norm(const DfSumP &a, f2x &h, f2x &l) {
  f2x L = a.L, C = a.C, f;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    two_sum2(L, a.V[j], L, f);
    C = add2(C, f);
  }
  f2x s, e;
  two_sum2(a.H, L, s, e);
  two_sum2(s, add2(e, C), h, l);
}

// Normalised (hi, lo) per lane of a paired accumulator.
__device__ __forceinline__ void acc2_norm(const DfAcc2 &a, f2x &h, f2x &l) {
  const f2x s = add2(a.H, a.L);
  const f2x bb = sub2(s, a.H);
  l = add2(sub2(a.H, sub2(s, bb)), sub2(a.L, bb));
  h = s;
}

// Packed double-float arithmetic on two lanes; the same operation sequences as df_add and
// df_mul.
__device__ __forceinline__ void df2_add(f2x ah, f2x al, f2x bh, f2x bl, f2x &rh, f2x &rl) {
  const f2x s = add2(ah, bh);
  const f2x bb = sub2(s, ah);
  f2x e = add2(sub2(ah, sub2(s, bb)), sub2(bh, bb));
  e = add2(e, add2(al, bl));
  rh = add2(s, e);
  rl = sub2(e, sub2(rh, s));
}
__device__ __forceinline__ void df2_sub(f2x ah, f2x al, f2x bh, f2x bl, f2x &rh, f2x &rl) {
  const f2x s = sub2(ah, bh);
  const f2x bb = sub2(s, ah);
  f2x e = sub2(sub2(ah, sub2(s, bb)), add2(bh, bb));
  e = add2(e, sub2(al, bl));
  rh = add2(s, e);
  rl = sub2(e, sub2(rh, s));
}
// The product is taken lane by lane with the scalar df_mul: a packed TwoProd (mul.rn.f32x2
// followed by fma.rn.f32x2 of the same operands against the negated product) was measured
// on this GPU to return the high-part product without its rounding error in some code
// shapes (relative error up to 2^-24), while the scalar sequence is exact.
__device__ __forceinline__ void df2_mul(f2x ah, f2x al, f2x bh, f2x bl, f2x &rh, f2x &rl) {
  const float2 a_h = upk2(ah), a_l = upk2(al), b_h = upk2(bh), b_l = upk2(bl);
  const float2 r0 = df_mul(make_float2(a_h.x, a_l.x), make_float2(b_h.x, b_l.x));
  const float2 r1 = df_mul(make_float2(a_h.y, a_l.y), make_float2(b_h.y, b_l.y));
  rh = pk2(r0.x, r1.x);
  rl = pk2(r0.y, r1.y);
}

// Lane a / lane b of a paired accumulator as a plain accumulator.
__device__ __forceinline__ DfAcc acc2_lane(const DfAcc2 &a, int lane) {
  const float2 h = upk2(a.H), l = upk2(a.L);
  return lane == 0 ? DfAcc{h.x, l.x} : DfAcc{h.y, l.y};
}

// 2^k as a float for -126 <= k <= 127.
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((uint32_t)(k + 127) << 23); }

// FP64 -> double-float with a power-of-two scale 2^-shift applied exactly, using integer
// instructions only: hi takes the leading 24 significant bits (truncated), lo the next 29
// bits rounded to FP32 (error <= 2^-48 |x|).  Zero and FP64 subnormals map to 0; results
// below the FP32 normal range keep FP32 gradual underflow.  Requires |x| 2^-shift < 2^127.
__device__ __forceinline__ float2 f64_to_df(double x, int shift) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t hi32 = (uint32_t)(b >> 32), lo32 = (uint32_t)b;
  const int e = (int)((hi32 >> 20) & 0x7ffu);
  if (e == 0) return make_float2(0.f, 0.f);
  const int E = e - 1023 - shift;                       // x 2^-shift = 1.f * 2^E
  const uint32_t sign = hi32 & 0x80000000u;
  const uint32_t m23 = ((hi32 & 0xfffffu) << 3) | (lo32 >> 29);
  const float one_m = __uint_as_float(0x3f800000u | m23);   // 1.m23 in [1, 2)
  const uint32_t rem = lo32 & 0x1fffffffu;                   // next 29 bits: rem * 2^-52
  float h, l;
  // scale in two exact steps so that every intermediate power of two is a normal float
  const int k1 = E > 0 ? (E > 126 ? 126 : E) : (E < -126 ? -126 : E);
  const int k2 = E - k1;
  h = __fmul_rn(__fmul_rn(one_m, pow2f(k1)), pow2f(k2 < -126 ? -126 : k2));
  l = __fmul_rn(__fmul_rn(__uint2float_rn(rem), pow2f(-52)), pow2f(k1));
  l = __fmul_rn(l, pow2f(k2 < -126 ? -126 : k2));
  if (sign) {
    h = -h;
    l = -l;
  }
  return make_float2(h, l);
}

// Exact FP32 -> FP64 bit pattern conversion with integer instructions (normal and
// subnormal floats), scaled by 2^shift.
__device__ __forceinline__ double f32_to_f64_scaled(float f, int shift) {
  uint32_t u = __float_as_uint(f);
  const uint32_t sign = u & 0x80000000u;
  uint32_t mag = u & 0x7fffffffu;
  if (mag == 0) return __longlong_as_double((long long)((uint64_t)sign << 32));
  int e = (int)(mag >> 23);
  uint32_t m = mag & 0x7fffffu;
  if (e == 0) {                 // subnormal: normalise
    int lz = __clz(m) - 8;      // leading zeros within the 23-bit field
    m = (m << (lz + 1)) & 0x7fffffu;
    e = 1 - (lz + 1);
  }
  const uint64_t E = (uint64_t)(e - 127 + 1023 + shift);
  const uint64_t bits = ((uint64_t)sign << 32) | (E << 52) | ((uint64_t)m << 29);
  return __longlong_as_double((long long)bits);
}

// Double-float -> FP64 (scaled by 2^shift): two exact conversions and one FP64 add.
__device__ __forceinline__ double df_to_f64(float2 v, int shift) {
  return f32_to_f64_scaled(v.x, shift) + f32_to_f64_scaled(v.y, shift);
}

}  // namespace hub
