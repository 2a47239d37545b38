// fxsum.h -- the FP64 neighbour sum of the constant-coefficient stencils in
// 64-bit fixed point (host and device; the host build serves the tests).
//
// On GB300 an FP64 add issues at 2 per clock per SM while integer operations
// issue at 64 or more, and the FP64 stencil sweep is bound by its FP64
// instructions, five of which are the neighbour sum's additions (3D).  The
// sum is therefore formed on the integer units: every operand's 53-bit
// significand, shifted 6 bits up, is aligned to the largest operand's
// exponent (bits below its unit 2^(emax - 1081) are dropped, toward zero),
// the signed 64-bit integers are added exactly, and the total is rounded
// to FP64 once (to nearest even, in integer operations) with the exponent
// of its unit (a normal number in the range checked).  Error: below K units
// of 2^(emax - 1081) from the dropped bits (subnormal operands lie below the
// unit) plus half an ulp of the result, i.e. at most K * 2^-58 * max|x_k| +
// 2^-53 |sum| -- tighter than the (K - 1) * 2^-53 * sum|x_k| bound of K - 1
// rounded FP64 additions.  Operands whose largest binade is outside
// [2^-964, 2^1019] (all zero, tiny, huge, Inf, NaN) take the plain FP64
// additions, out of line.
#pragma once

#include <stdint.h>
#include <string.h>

#include "plcg_internal.h"

namespace plcg {

PLCG_HD inline uint64_t fx_bits(double x)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    memcpy(&u, &x, sizeof u);
    return u;
#endif
}

PLCG_HD inline double fx_from_bits(uint64_t u)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double x;
    memcpy(&x, &u, sizeof x);
    return x;
#endif
}

PLCG_HD inline int fx_clz64(uint64_t u)   // u != 0
{
#ifdef __CUDA_ARCH__
    return __clzll((long long)u);
#else
    return __builtin_clzll(u);
#endif
}

#ifdef __CUDACC__
#define PLCG_FX_NOINLINE __noinline__
#else
#define PLCG_FX_NOINLINE __attribute__((noinline))
#endif

// The plain FP64 additions of the out-of-range case, out of line: kept off
// the common path (not evaluated alongside it).
template <int K>
struct FxOperands {
    double v[K];
};

template <int K>
PLCG_HD PLCG_FX_NOINLINE double fx_plain_sum(FxOperands<K> x)
{
    double s = x.v[0];
#pragma unroll
    for (int k = 1; k < K; ++k) s += x.v[k];
    return s;
}

constexpr int kFxShift = 6;                        // significand headroom: 2^58 <= m < 2^59
constexpr int kFxUnitBias = 1075 + kFxShift;       // unit of the sum: 2^(emax - kFxUnitBias)
constexpr int kFxEmaxLo = kFxUnitBias - 1022;      // |acc| >= 1: result exponent >= 1
constexpr int kFxEmaxHi = 2046 + kFxUnitBias - 1085;   // |acc| < 2^62, rounded up to 2^62 at most

// Sum of the K <= 8 values x[0..K-1] (see above).
template <int K>
PLCG_HD inline double fx_sum(const double (&x)[K])
{
    static_assert(K >= 1 && K <= 8, "K * 2^59 must stay below 2^62");
    uint64_t b[K];
    int emax = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        b[k] = fx_bits(x[k]);
        const int e = (int)((b[k] >> 52) & 0x7ff);
        emax = e > emax ? e : emax;
    }
    if (__builtin_expect(emax < kFxEmaxLo || emax > kFxEmaxHi, 0)) {
        FxOperands<K> o;
#pragma unroll
        for (int k = 0; k < K; ++k) o.v[k] = x[k];
        return fx_plain_sum<K>(o);
    }
    int64_t acc = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int e = (int)((b[k] >> 52) & 0x7ff);
        // the significand with its implicit bit at bit 63, shifted down to
        // the unit: (M << 11) >> (11 - kFxShift + emax - e).  Zeros and
        // subnormals (e = 0) shift by more than 63 since emax >= kFxEmaxLo,
        // and add nothing (a subnormal is below the unit)
        const uint64_t t = (b[k] << 11) | (1ull << 63);
        const int sh = 11 - kFxShift + emax - e;
        const uint64_t m = sh < 64 ? (t >> sh) : 0ull;
        acc += (b[k] >> 63) ? -(int64_t)m : (int64_t)m;
    }
    if (acc == 0) return 0.0;
    // the one rounding, on the integer units as well (an int64 -> FP64
    // conversion issues on the FP64 pipe): normalise |acc| to bit 63, keep
    // 53 bits, round to nearest even on the 11 below; a carry out of the
    // 53 bits moves into the exponent field by the final add
    const uint64_t neg = (uint64_t)acc >> 63;
    const uint64_t mag = neg ? (uint64_t)0 - (uint64_t)acc : (uint64_t)acc;
    const int lz = fx_clz64(mag);              // 2 <= lz <= 63
    const uint64_t nrm = mag << lz;
    uint64_t sig = nrm >> 11;                  // 2^52 <= sig < 2^53
    const uint64_t rem = nrm & 0x7ffull;
    sig += (rem > 0x400ull || (rem == 0x400ull && (sig & 1ull))) ? 1ull : 0ull;
    // |sum| = sig * 2^(11 - lz) * 2^(emax - kFxUnitBias) = sig * 2^(E - 1075)
    const int E = emax - lz + 11 - kFxUnitBias + 1075;
    return fx_from_bits((neg << 63) + ((uint64_t)(E - 1) << 52) + sig);
}

}  // namespace plcg
