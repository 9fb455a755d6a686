// Device modular arithmetic on 64-bit words, primes 2^32 < q < 2^61.
//
//  * Shoup multiplication by a fixed operand w with companion
//    w' = floor(w * 2^64 / q): result in [0, 2q) for any 64-bit input
//    (Shoup; bound as in Harvey, "Faster arithmetic for number-theoretic
//    transforms", 2014).
//  * Barrett reduction of a product x < q^2 with mu = floor(2^(2b) / q),
//    b = bit length of q (Barrett 1986): quotient estimate
//    floor(floor(x / 2^(b-1)) * mu / 2^(b+1)), remainder in [0, 3q).
#pragma once
#include <cstdint>

namespace hedap {

typedef uint64_t u64;

struct PrimeDev {  // per-prime constants used by the kernels
  u64 q;
  u64 mu;       // floor(2^(2b) / q)
  int b;        // bit length of q
  int pad;
};

// High 64 bits of x * y, exact, from 32-bit pieces: the middle column (hi(x0 y0) + lo(x0 y1) +
// lo(x1 y0)) is summed only for its carries, then the upper columns with carry chains.  Eight
// 32-bit multiply-adds; measured faster than four 32 x 32 -> 64 products with 64-bit partial sums.
__device__ __forceinline__ u64 mulhi64(u64 x, u64 y) {
  u64 h;
  asm("{\n\t"
      ".reg .u32 x0, x1, y0, y1, t0, t1, t2, h0, h1;\n\t"
      "mov.b64 {x0, x1}, %1;\n\t"
      "mov.b64 {y0, y1}, %2;\n\t"
      "mul.hi.u32 t0, x0, y0;\n\t"
      "mad.lo.cc.u32 t0, x0, y1, t0;\n\t"
      "madc.hi.u32 t1, x0, y1, 0;\n\t"
      "mad.lo.cc.u32 t0, x1, y0, t0;\n\t"
      "madc.hi.cc.u32 t1, x1, y0, t1;\n\t"
      "addc.u32 t2, 0, 0;\n\t"
      "mad.lo.cc.u32 h0, x1, y1, t1;\n\t"
      "madc.hi.u32 h1, x1, y1, t2;\n\t"
      "mov.b64 %0, {h0, h1};\n\t"
      "}"
      : "=l"(h)
      : "l"(x), "l"(y));
  return h;
}
// x * w - floor(x * wp / 2^64) * q  mod 2^64, in [0, 2q): the quotient qh = mulhi64(x, wp), then
// x * w + qh * (2^64 - q) mod 2^64 in two wide and four low multiply-adds.
__device__ __forceinline__ u64 shoup_mul_lazy(u64 x, u64 w, u64 wp, u64 q) {
  const u64 nq = 0 - q, qh = mulhi64(x, wp);
  u64 r;
  asm("{\n\t"
      ".reg .u32 x0, x1, a0, a1, n0, n1, h0, h1, r0, r1;\n\t"
      ".reg .u64 p;\n\t"
      "mov.b64 {x0, x1}, %1;\n\t"
      "mov.b64 {a0, a1}, %2;\n\t"
      "mov.b64 {n0, n1}, %4;\n\t"
      "mov.b64 {h0, h1}, %3;\n\t"
      "mul.wide.u32 p, a0, x0;\n\t"
      "mad.wide.u32 p, h0, n0, p;\n\t"
      "mov.b64 {r0, r1}, p;\n\t"
      "mad.lo.u32 r1, a0, x1, r1;\n\t"
      "mad.lo.u32 r1, a1, x0, r1;\n\t"
      "mad.lo.u32 r1, h0, n1, r1;\n\t"
      "mad.lo.u32 r1, h1, n0, r1;\n\t"
      "mov.b64 %0, {r0, r1};\n\t"
      "}"
      : "=l"(r)
      : "l"(x), "l"(w), "l"(qh), "l"(nq));
  return r;
}
__device__ __forceinline__ u64 shoup_mul(u64 x, u64 w, u64 wp, u64 q) {
  u64 r = shoup_mul_lazy(x, w, wp, q);
  return r >= q ? r - q : r;
}
__device__ __forceinline__ u64 barrett_reduce(u64 lo, u64 hi, const PrimeDev& p) {
  // t = floor(x / 2^(b-1)) (< 2^(b+1)), qhat = floor(t * mu / 2^(b+1))
  int s = p.b - 1;
  u64 t = (lo >> s) | (hi << (64 - s));
  u64 plo = t * p.mu, phi = mulhi64(t, p.mu);
  int s2 = p.b + 1;
  u64 qhat = (plo >> s2) | (phi << (64 - s2));
  u64 r = lo - qhat * p.q;
  if (r >= p.q) r -= p.q;
  if (r >= p.q) r -= p.q;
  return r;
}
__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, const PrimeDev& p) {
  return barrett_reduce(a * b, mulhi64(a, b), p);
}
__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) {
  u64 s = a + b;
  return s >= q ? s - q : s;
}
__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) {
  return a >= b ? a - b : a + q - b;
}
// 128-bit accumulator helpers for lazy sums of products
struct Acc128 {
  u64 lo, hi;
};
// acc += a * b as four 32-bit columns with carry chains (the caller keeps the sum below 2^128)
__device__ __forceinline__ void mac128(Acc128& acc, u64 a, u64 b) {
  asm("{\n\t"
      ".reg .u32 a0, a1, b0, b1, c0, c1, c2, c3;\n\t"
      "mov.b64 {a0, a1}, %2;\n\t"
      "mov.b64 {b0, b1}, %3;\n\t"
      "mov.b64 {c0, c1}, %0;\n\t"
      "mov.b64 {c2, c3}, %1;\n\t"
      "mad.lo.cc.u32 c0, a0, b0, c0;\n\t"
      "madc.hi.cc.u32 c1, a0, b0, c1;\n\t"
      "madc.lo.cc.u32 c2, a1, b1, c2;\n\t"
      "madc.hi.u32 c3, a1, b1, c3;\n\t"
      "mad.lo.cc.u32 c1, a0, b1, c1;\n\t"
      "madc.hi.cc.u32 c2, a0, b1, c2;\n\t"
      "addc.u32 c3, c3, 0;\n\t"
      "mad.lo.cc.u32 c1, a1, b0, c1;\n\t"
      "madc.hi.cc.u32 c2, a1, b0, c2;\n\t"
      "addc.u32 c3, c3, 0;\n\t"
      "mov.b64 %0, {c0, c1};\n\t"
      "mov.b64 %1, {c2, c3};\n\t"
      "}"
      : "+l"(acc.lo), "+l"(acc.hi)
      : "l"(a), "l"(b));
}
// reduce an arbitrary 128-bit value: hi is first brought below q, then the
// value hi'*2^64 + lo < q*2^64 < q^2 * 2^(64-b) ... is reduced in two Barrett
// steps on 2^64-aligned halves: x = hi' * 2^64 + lo = (hi' * r64 + lo) mod q,
// with r64 = 2^64 mod q.
__device__ __forceinline__ u64 reduce128(Acc128 x, const PrimeDev& p, u64 r64, u64 r64p) {
  u64 hi = x.hi;
  if (hi >= p.q) hi = barrett_reduce(hi, 0, p);           // hi < 2^64 <= q^2 for b >= 32
  u64 a = shoup_mul(hi, r64, r64p, p.q);                  // hi * 2^64 mod q
  u64 lo = x.lo;
  u64 lr = barrett_reduce(lo, 0, p);                      // lo < 2^64 <= q^2
  return add_mod(a, lr, p.q);
}

}  // namespace hedap
