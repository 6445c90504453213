// chanfs_f64emu.cuh -- IEEE-754 binary64 addition and subtraction on the
// integer units, bit for bit the round-to-nearest-even result of the FP64
// pipe.
//
// The FP64 transforms are bound by the FP64 pipe: GB300 executes two FP64
// lanes per SM per clock, one warp instruction every 16 clocks, while the
// same SM issues four warp instructions per clock to its integer and FP32
// pipes.  A butterfly pair (a + b, a - b) computed here costs a few dozen
// integer and logic instructions instead of two FP64 instructions, so a
// transform that moves part of its additions here runs both kinds of units
// at once.  The results are the FP64 pipe's, so a kernel gives the same bits
// whichever additions it moves.
//
// The arithmetic follows the definition of binary64 addition (IEEE 754,
// round to nearest, ties to even): align the smaller magnitude to the
// larger's exponent, keep the bits shifted out as a sticky bit, add or
// subtract the significands, normalise, round.  The fast path takes operands
// whose biased exponents lie in [64, 2045]; there no result can be subnormal
// or overflow (a difference of such operands is zero or at least 2^-1011 in
// magnitude, a sum below 2^1024 - 2^970), and an exact zero difference is +0
// as the standard requires.  Any other operand (zero, subnormal, tiny, huge,
// infinity, NaN) takes the FP64 pipe.
#pragma once

#include <stdint.h>
#include <string.h>

namespace chanfs {

__host__ __device__ __forceinline__ uint64_t emu_bits(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  memcpy(&u, &x, sizeof u);
  return u;
#endif
}

__host__ __device__ __forceinline__ double emu_double(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  memcpy(&x, &u, sizeof x);
  return x;
#endif
}

// Leading zeros of a nonzero 64-bit word.
__host__ __device__ __forceinline__ int emu_clz(uint64_t v) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)v);
#else
  return __builtin_clzll(v);
#endif
}

constexpr uint64_t kEmuSign = 0x8000000000000000ull;
constexpr uint64_t kEmuFrac = 0x000fffffffffffffull;
constexpr uint64_t kEmuHidden = 0x0010000000000000ull;

// A significand m with its leading bit at bit 62 (the 53 kept bits at 62..10,
// the 10 bits below them ending in a sticky bit) rounded to nearest even and
// packed with biased exponent e: adding 0x1ff plus the last kept bit carries
// into the kept bits exactly when the dropped part exceeds half a unit, or
// equals it and the kept part is odd.  The hidden bit of the rounded value
// adds one to the exponent field (two when rounding carried to 2^53, which
// is then the next binade with a zero fraction).
__host__ __device__ __forceinline__ uint64_t emu_round_pack(uint64_t m, int e) {
  const uint64_t r = (m + 0x1ffull + ((m >> 10) & 1ull)) >> 10;
  return ((uint64_t)(e - 1) << 52) + r;
}

// |X| + |Y| and |X| - |Y| as binary64 magnitudes, for magnitudes X >= Y
// (sign bits clear) with biased exponents in [64, 2045].
__host__ __device__ __forceinline__ void emu_addsub_mag(uint64_t X, uint64_t Y, uint64_t& sum,
                                                        uint64_t& dif) {
  const int ex = (int)(X >> 52), ey = (int)(Y >> 52);
  const uint64_t mx = ((X & kEmuFrac) | kEmuHidden) << 10;
  const uint64_t my = ((Y & kEmuFrac) | kEmuHidden) << 10;
  const int d = min(ex - ey, 63);
  const uint64_t ys = my >> d;
  const uint64_t yst = ys | (uint64_t)((ys << d) != my);  // sticky bit of what was shifted out
  // sum: the leading bit lands on bit 62 or 63
  uint64_t a = mx + yst;
  const int up = (int)(a >> 63);
  a = (a >> up) | (a & (uint64_t)up);
  sum = emu_round_pack(a, ex + up);
  // difference: leading bit on bit 62 or below (far below only when d <= 1,
  // where nothing was shifted out and the difference is exact)
  const uint64_t b = mx - yst;
  const int sh = b ? emu_clz(b) - 1 : 0;
  dif = b ? emu_round_pack(b << sh, ex - sh) : 0ull;
}

// Whether both operands take the integer path: biased exponents in [64, 2045].
__host__ __device__ __forceinline__ bool emu_fast(uint64_t ua, uint64_t ub) {
  const uint32_t ea = (uint32_t)(ua >> 52) & 0x7ffu, eb = (uint32_t)(ub >> 52) & 0x7ffu;
  return (ea - 64u) <= 1981u && (eb - 64u) <= 1981u;
}

// s = a + b and d = a - b, each exactly as the FP64 pipe rounds it.  With X
// the operand of larger magnitude and Y the other, both X + Y and X - Y take
// X's sign (or are +0): X + Y has magnitude |X| + |Y| when the signs agree,
// else |X| - |Y|, and X - Y the other one.  a + b = X + Y, and
// a - b = X - Y, negated when X is b.
__host__ __device__ __forceinline__ void f64_addsub(double a, double b, double& s, double& d) {
  const uint64_t ua = emu_bits(a), ub = emu_bits(b);
  if (!emu_fast(ua, ub)) {
    s = a + b;
    d = a - b;
    return;
  }
  const uint64_t ma = ua & ~kEmuSign, mb = ub & ~kEmuSign;
  const bool sw = mb > ma;
  const uint64_t X = sw ? mb : ma, Y = sw ? ma : mb;
  const uint64_t sx = (sw ? ub : ua) & kEmuSign;
  uint64_t madd, msub;
  emu_addsub_mag(X, Y, madd, msub);
  const bool same = ((ua ^ ub) & kEmuSign) == 0;
  const uint64_t ps = same ? madd : msub;
  const uint64_t qs = same ? msub : madd;
  s = emu_double(ps ? (ps | sx) : 0ull);
  d = emu_double(qs ? (qs | (sw ? sx ^ kEmuSign : sx)) : 0ull);
}

}  // namespace chanfs
