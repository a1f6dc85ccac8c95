// Floating-point primitives of the enhanced Kogbetliantz 2x2 SVD (arXiv 2407.13116, Sect. 2)
// for sm_103a.  Everything here is exact or correctly rounded (round to nearest, ties to
// even, gradual underflow); the kernels are compiled with -ftz=false -prec-div=true
// -prec-sqrt=true --fmad=false, so the only fused operations are explicit fma calls.
//
// GB300 has a narrow FP64 pipe (about 2 DFMA per clock per SM), so the exact steps that
// do not need FP64 arithmetic -- exponent extraction, (e,f) renormalisation, power-of-two
// scaling, the rounding decision of hypot and the binary128 emulation of eq. (EXT) -- run
// on the integer pipes.
#pragma once
#include <cstdint>

namespace k2 {

typedef unsigned __int128 u128;

constexpr uint64_t D_MANT = 0x000FFFFFFFFFFFFFull;
constexpr uint64_t D_HID = 0x0010000000000000ull;
constexpr uint64_t D_SIGN = 0x8000000000000000ull;
constexpr uint32_t F_MANT = 0x007FFFFFu;
constexpr uint32_t F_HID = 0x00800000u;
constexpr uint32_t F_SIGN = 0x80000000u;

__device__ __forceinline__ uint64_t dbits(double x) { return (uint64_t)__double_as_longlong(x); }
__device__ __forceinline__ double dfrom(uint64_t b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ uint32_t fbits(float x) { return (uint32_t)__float_as_uint(x); }
__device__ __forceinline__ float ffrom(uint32_t b) { return __uint_as_float(b); }

__device__ __forceinline__ int clz128(u128 x)
{
    uint64_t hi = (uint64_t)(x >> 64), lo = (uint64_t)x;
    return hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
}

// ---------------------------------------------------------------------------------------
// IEEE comparisons for operands that are never NaN: for double on the bit patterns (the
// integer pipes; the FP64 pipe is the scarce one), for float as native FP32 compares (3-4%
// faster for the FP32 kernels, same results).  gt0/lt0 follow IEEE (+-0 is neither);
// pos_lt / pos_eq are for non-negative operands (+0 .. +inf); eq0 is true for +0 and -0.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ bool lt0(double x) { int64_t b = (int64_t)dbits(x); return b < 0 && (b << 1) != 0; }
__device__ __forceinline__ bool lt0(float x) { return x < 0.0f; }
__device__ __forceinline__ bool gt0(double x) { return (int64_t)dbits(x) > 0; }
__device__ __forceinline__ bool gt0(float x) { return x > 0.0f; }
__device__ __forceinline__ bool eq0(double x) { return (dbits(x) << 1) == 0; }
__device__ __forceinline__ bool eq0(float x) { return x == 0.0f; }
__device__ __forceinline__ bool pos_lt(double a, double b) { return dbits(a) < dbits(b); }
__device__ __forceinline__ bool pos_lt(float a, float b) { return a < b; }
__device__ __forceinline__ bool pos_eq(double a, double b) { return dbits(a) == dbits(b); }
__device__ __forceinline__ bool pos_eq(float a, float b) { return a == b; }
__device__ __forceinline__ bool is_inf(double x) { return (dbits(x) << 1) == (0x7FFull << 53); }
__device__ __forceinline__ bool is_inf(float x) { return fabsf(x) == __int_as_float(0x7f800000); }
__device__ __forceinline__ bool is_fin(double x) { return ((dbits(x) >> 52) & 0x7FF) != 0x7FF; }
__device__ __forceinline__ bool is_fin(float x) { return fabsf(x) <= 0x1.fffffep127f; }
// |a| < |b| for finite, non-NaN operands
__device__ __forceinline__ bool abs_lt(double a, double b) { return (dbits(a) << 1) < (dbits(b) << 1); }
__device__ __forceinline__ bool abs_lt(float a, float b) { return fabsf(a) < fabsf(b); }
// -0 -> +0, anything else unchanged
__device__ __forceinline__ double absv(double x) { return dfrom(dbits(x) & ~D_SIGN); }
__device__ __forceinline__ float absv(float x) { return fabsf(x); }
__device__ __forceinline__ double unneg0(double x) { uint64_t b = dbits(x); return dfrom(b == D_SIGN ? 0 : b); }
__device__ __forceinline__ float unneg0(float x) { uint32_t b = fbits(x); return ffrom(b == F_SIGN ? 0u : b); }

// ---------------------------------------------------------------------------------------
// Per-type traits: exponent/mantissa split, exact scaling, constants.
// For x != 0 finite: e = floor(lg|x|) (also for subnormals) and f = x 2^-e, 1 <= |f| < 2.
// ---------------------------------------------------------------------------------------
template <typename T> struct fpt;

template <> struct fpt<double> {
    typedef uint64_t bits_t;
    static constexpr int P = 53, EMU = -1022, ENU = 1023;
    __device__ static __forceinline__ double eps() { return 0x1p-53; }
    __device__ static __forceinline__ double nu() { return 0x1.fffffffffffffp1023; }
    __device__ static __forceinline__ double mu() { return 0x1p-1022; }

    // (e, f) of x != 0
    __device__ static __forceinline__ void split(double x, int &e, double &f)
    {
        uint64_t b = dbits(x), m = b & D_MANT;
        int E = (int)((b >> 52) & 0x7FF);
        if (E == 0) {
            int sh = __clzll((long long)m) - 11;
            e = -1022 - sh;
            m = (m << sh) & D_MANT;
        } else {
            e = E - 1023;
        }
        f = dfrom((b & D_SIGN) | (1023ull << 52) | m);
    }
    __device__ static __forceinline__ int expo(double x) { int e; double f; split(x, e, f); return e; }
    // f * 2^e rounded once; f = 0 or 1 <= |f| < 2
    __device__ static __forceinline__ double ldexp_rn(double f, int e)
    {
        if (eq0(f)) return f;
        uint64_t b = dbits(f), keep = b & (D_SIGN | D_MANT);
        if (e > 1023) return dfrom((b & D_SIGN) | (0x7FFull << 52));
        if (e >= -1022) return dfrom(keep | ((uint64_t)(e + 1023) << 52));
        if (e < -1100) return dfrom(b & D_SIGN);
        // subnormal result: one rounding, by a product with a normal power of two
        double y = dfrom(keep | ((uint64_t)(e + 600 + 1023) << 52));
        return y * 0x1p-600;
    }
    // x 2^s rounded once, any finite x
    __device__ static __forceinline__ double scale(double x, int s)
    {
        if (eq0(x)) return x;
        int e; double f; split(x, e, f);
        return ldexp_rn(f, e + s);
    }
};

template <> struct fpt<float> {
    typedef uint32_t bits_t;
    static constexpr int P = 24, EMU = -126, ENU = 127;
    __device__ static __forceinline__ float eps() { return 0x1p-24f; }
    __device__ static __forceinline__ float nu() { return 0x1.fffffep127f; }
    __device__ static __forceinline__ float mu() { return 0x1p-126f; }

    __device__ static __forceinline__ void split(float x, int &e, float &f)
    {
        uint32_t b = fbits(x), m = b & F_MANT;
        int E = (int)((b >> 23) & 0xFF);
        if (E == 0) {
            int sh = __clz((int)m) - 8;
            e = -126 - sh;
            m = (m << sh) & F_MANT;
        } else {
            e = E - 127;
        }
        f = ffrom((b & F_SIGN) | (127u << 23) | m);
    }
    __device__ static __forceinline__ int expo(float x) { int e; float f; split(x, e, f); return e; }
    __device__ static __forceinline__ float ldexp_rn(float f, int e)
    {
        if (eq0(f)) return f;
        uint32_t b = fbits(f), keep = b & (F_SIGN | F_MANT);
        if (e > 127) return ffrom((b & F_SIGN) | (0xFFu << 23));
        if (e >= -126) return ffrom(keep | ((uint32_t)(e + 127) << 23));
        if (e < -160) return ffrom(b & F_SIGN);
        float y = ffrom(keep | ((uint32_t)(e + 64 + 127) << 23));
        return y * 0x1p-64f;
    }
    __device__ static __forceinline__ float scale(float x, int s)
    {
        if (eq0(x)) return x;
        int e; float f; split(x, e, f);
        return ldexp_rn(f, e + s);
    }
};

// ---------------------------------------------------------------------------------------
// Correctly rounded binary64 division on the integer pipes (round to nearest, ties to
// even, gradual underflow).  The FP64 pipe of sm_103 divides at about one ninth of its fma
// rate, while 32-bit integer multiply-adds issue at 16-62 per clock per SM, so the quotient
// is formed by long division in integers:
//   * the mantissas A, B (53-bit integers, subnormals normalised) are brought to
//     B <= A < 2B by one shift, so the quotient is 1.f with e = e_a - e_b (- 1);
//   * three 19-bit fraction digits follow; each is estimated as
//     trunc((r >> 29) * (2^19 / (B >> 29))) with one FP32 reciprocal of the 24 leading bits of
//     B.  The estimate is within 0.19 of r 2^19 / B (relative errors below 2^-22 and a
//     truncation of r below 2^48 / B < 1/16 of a digit), so one correction by +-1 against
//     the exact remainder gives the digit.  The remainder fits in 2^54, so its low 64 bits
//     (wrapping arithmetic) are exact;
//   * the 58-bit quotient and the sticky remainder are rounded to 53 bits, or to the
//     quantum 2^-1074 when the result is subnormal; overflow gives infinity.
// Zero, infinite and NaN operands give the IEEE results by selection (no FP64 instruction).
//
// div_rn, hypot_cr and ext_num_div are kept out of line: the 2x2 kernel calls them from a
// dozen divergent branches, and with every call site inlined the FP64 kernel ran 2.9 times
// (FP32: 1.1 times) slower on matrices of mixed zero pattern and wide exponent range
// (measured on a GB300; the instruction stream grows with each copy, and divergent warps
// fetch from all of them).  One shared body per function keeps the executed code small.
// The out-of-line bodies take and return bit patterns (uint64_t): on sm_103 a call that
// passes doubles spends FP64-pipe instructions on moving them (2 per call, measured), and
// the FP64 pipe is the scarce one.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double div_rn_body(double a, double b)
{
    const uint64_t ab = dbits(a), bb = dbits(b);
    const uint32_t Ea = (uint32_t)(ab >> 52) & 0x7FF, Eb = (uint32_t)(bb >> 52) & 0x7FF;
    if (Ea == 0x7FF || Eb == 0x7FF || (ab << 1) == 0 || (bb << 1) == 0) {
        // zero, infinite or NaN operands: IEEE results by selection
        const uint64_t sg = (ab ^ bb) & D_SIGN;
        const bool an = (ab << 1) > (0x7FFull << 53), bn = (bb << 1) > (0x7FFull << 53);
        const bool ai = (ab << 1) == (0x7FFull << 53), bi = (bb << 1) == (0x7FFull << 53);
        const bool az = (ab << 1) == 0, bz = (bb << 1) == 0;
        if (an || bn || (az && bz) || (ai && bi)) return dfrom(0x7FF8000000000000ull);
        if (az || bi) return dfrom(sg);
        return dfrom(sg | (0x7FFull << 52));
    }
    uint64_t A = ab & D_MANT, B = bb & D_MANT;
    int ea, eb;
    if (Ea) { A |= D_HID; ea = (int)Ea - 1023; } else { int sh = __clzll((long long)A) - 11; A <<= sh; ea = -1022 - sh; }
    if (Eb) { B |= D_HID; eb = (int)Eb - 1023; } else { int sh = __clzll((long long)B) - 11; B <<= sh; eb = -1022 - sh; }
    int e = ea - eb;
    if (A < B) { A <<= 1; e -= 1; }
    const float rf = __frcp_rn(__uint2float_rz((uint32_t)(B >> 29))) * 524288.0f;      // 2^19 / (B >> 29)
    uint64_t r = A - B, q = 1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        uint32_t d = __float2uint_rz(__uint2float_rz((uint32_t)(r >> 29)) * rf);
        int64_t rem = (int64_t)((r << 19) - (uint64_t)d * B);
        if (rem < 0) { d -= 1; rem += (int64_t)B; }
        else if (rem >= (int64_t)B) { d += 1; rem -= (int64_t)B; }
        r = (uint64_t)rem;
        q = (q << 19) | d;
    }
    const uint64_t sign = (ab ^ bb) & D_SIGN;
    const bool sticky = r != 0;
    if (e >= -1022) {                                       // normal: q in [2^57, 2^58) -> 53 bits
        uint64_t m = q >> 5;
        const bool rb = (q >> 4) & 1, st = sticky || (q & 15) != 0;
        if (rb && (st || (m & 1))) ++m;
        if (m >> 53) { m >>= 1; ++e; }
        if (e > 1023) return dfrom(sign | (0x7FFull << 52));
        return dfrom(sign | ((uint64_t)(e + 1023) << 52) | (m & D_MANT));
    }
    const int k = -1017 - e;                                // bits of q below the quantum 2^-1074
    if (k > 63) return dfrom(sign);
    uint64_t m = q >> k;
    const bool rb = (q >> (k - 1)) & 1, st = sticky || (q & ((1ull << (k - 1)) - 1)) != 0;
    if (rb && (st || (m & 1))) ++m;
    return dfrom(sign | m);                                 // m <= 2^52: subnormal or 2^-1022
}

static __device__ __noinline__ uint64_t div_rn_bits(uint64_t a, uint64_t b) { return dbits(div_rn_body(dfrom(a), dfrom(b))); }
__device__ __forceinline__ double div_rn(double a, double b) { return dfrom(div_rn_bits(dbits(a), dbits(b))); }

// The FP64 divider's correctly rounded quotient, out of line: one copy of the division
// sequence however many call sites use it (bit patterns in and out, as div_rn).
static __device__ __noinline__ uint64_t fdiv_rn_bits(uint64_t a, uint64_t b) { return dbits(__ddiv_rn(dfrom(a), dfrom(b))); }
__device__ __forceinline__ double fdiv_rn(double a, double b) { return dfrom(fdiv_rn_bits(dbits(a), dbits(b))); }

// the method's divisions: binary64 on the integer pipes, binary32 on the FP32 pipe
__device__ __forceinline__ double qdiv(double a, double b) { return div_rn(a, b); }
__device__ __forceinline__ float qdiv(float a, float b) { return a / b; }
// the same quotient with the binary64 body inlined at the call site, for a division that is
// the only one of its kernel half (no call, no shared body to fetch)
__device__ __forceinline__ double qdiv_inl(double a, double b) { return div_rn_body(a, b); }
__device__ __forceinline__ float qdiv_inl(float a, float b) { return a / b; }

// ---------------------------------------------------------------------------------------
// Exponent-"mantissa" pairs (Sect. 2): w = f 2^e with 1 <= |f| < 2, or (0, 0).
// ---------------------------------------------------------------------------------------
template <typename T> struct ef { int e; T f; };

template <typename T> __device__ __forceinline__ ef<T> ef_of(T x)
{
    ef<T> w;
    if (eq0(x)) { w.e = 0; w.f = T(0); }
    else fpt<T>::split(x, w.e, w.f);
    return w;
}
template <typename T> __device__ __forceinline__ T ef_fl(ef<T> w) { return fpt<T>::ldexp_rn(w.f, w.e); }

// eq. (binary): x (.) y; the mantissa product lies in [1,4)
// Renormalise a product in [1,4) or a quotient in (1/2,2) (or 0) to (e, f), 1 <= |f| < 2, by
// moving the binary exponent of z (exact, integer pipes).
__device__ __forceinline__ void renorm(double z, int e, int &eo, double &fo)
{
    uint64_t b = dbits(z);
    int E = (int)((b >> 52) & 0x7FF);
    if (E == 0) { eo = 0; fo = 0.0; return; }          // only z = 0 occurs here
    eo = e + (E - 1023);
    fo = dfrom((b & ~(0x7FFull << 52)) | (1023ull << 52));
}
__device__ __forceinline__ void renorm(float z, int e, int &eo, float &fo)
{
    uint32_t b = fbits(z);
    int E = (int)((b >> 23) & 0xFF);
    if (E == 0) { eo = 0; fo = 0.0f; return; }
    eo = e + (E - 127);
    fo = ffrom((b & ~(0xFFu << 23)) | (127u << 23));
}
template <typename T> __device__ __forceinline__ ef<T> ef_mul(ef<T> x, ef<T> y)
{
    ef<T> w;
    renorm(x.f * y.f, x.e + y.e, w.e, w.f);
    return w;
}
// eq. (binary): x (/) y; the mantissa quotient lies in (1/2, 2)
template <typename T> __device__ __forceinline__ ef<T> ef_div(ef<T> x, ef<T> y)
{
    ef<T> w;
    renorm(qdiv(x.f, y.f), x.e - y.e, w.e, w.f);
    return w;
}
// eq. (unary): 2^c (.) x
template <typename T> __device__ __forceinline__ ef<T> ef_pow2(int c, ef<T> x)
{
    if (!eq0(x.f)) x.e += c;
    return x;
}
// eq. (prec) for the non-negative values that occur here (sign(f) is 0 or 1)
template <typename T> __device__ __forceinline__ bool ef_prec(ef<T> x, ef<T> y)
{
    int sx = eq0(x.f) ? 0 : 1, sy = eq0(y.f) ? 0 : 1;
    if (sx != sy) return sx < sy;
    return (x.e < y.e) || ((x.e == y.e) && pos_lt(x.f, y.f));
}
// eq. (plus), x, y > 0 finite
template <typename T> __device__ __forceinline__ ef<T> ef_plus(T x, T y)
{
    T z = x + y;
    if (is_fin(z)) return ef_of(z);
    z = x * T(0.5) + y * T(0.5);
    ef<T> w = ef_of(z);
    w.e += 1;
    return w;
}
// eq. (minus), x, y > 0 finite; c = e_mu + p - 1 - min(e_x, e_y) (Lemma 2.4)
template <typename T> __device__ __forceinline__ ef<T> ef_minus(T x, T y)
{
    ef<T> w;
    if (pos_eq(x, y)) { w.e = 0; w.f = T(0); return w; }
    T z = x - y;
    if (!abs_lt(z, fpt<T>::mu())) return ef_of(z);
    int ex = fpt<T>::expo(x), ey = fpt<T>::expo(y);
    int c = fpt<T>::EMU + fpt<T>::P - 1 - (ex < ey ? ex : ey);
    z = fpt<T>::scale(x, c) - fpt<T>::scale(y, c);
    w = ef_of(z);
    if (!eq0(w.f)) w.e -= c;
    return w;
}

// ---------------------------------------------------------------------------------------
// floor(sqrt(X)) for an integer X in [2^110, 2^113), and the remainder X - floor(sqrt(X))^2,
// on the integer pipes (Newton's method for the square root):
//   * s0 = sqrt(X) (1 + e), |e| < 2^-21.4, from the FP32 reciprocal square root y of the
//     leading 31 bits of X (rsqrtf is within 2 ulp); Y = y 2^45 ~ 2^86 / sqrt(X) as a
//     32-bit integer;
//   * two corrections s <- s + (X - s^2) / (2 s) ~ s + R Y 2^-87: the residual R is exact
//     in 128-bit integers, its leading 31 bits times Y is one 32x32->64-bit product.  Error
//     bounds: |s1 - sqrt X| < 2^14.2 (Newton's quadratic term e0^2 / 2 sqrt X) + 2^13.5
//     (Y's relative error times |R0| / 2 sqrt X < 2^35.1) + 2^6 (R0 truncated to 31 bits) +
//     1 < 2^14.9, then |s2 - sqrt X| < 1/2 + 2^-6.7 + 2^-13;
//   * floor(sqrt X) is s2 or s2 - 1, decided by the sign of X - s2^2.
// No conversion involves a 64-bit type (those run on the FP64 pipe).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t isqrt113(u128 X, u128 &rem)
{
    const float xf = __uint2float_rz((uint32_t)(X >> 82));           // [2^28, 2^31)
    const float y = rsqrtf(xf);                                       // 2^41 / sqrt(X)
    const int64_t Y = (int64_t)__float2uint_rn(y * 0x1p45f);          // (2^29.5, 2^31]
    uint64_t s = (uint64_t)__float2uint_rn(xf * y * 0x1p9f) << 32;
    __int128 R = (__int128)(X - (u128)s * s);                         // |R| < 2^92.6
    s += (uint64_t)(((int64_t)(int32_t)(int64_t)(R >> 62) * Y) >> 25);
    R = (__int128)(X - (u128)s * s);                                  // |R| < 2^72.5
    s += (uint64_t)(((int64_t)(int32_t)(int64_t)(R >> 43) * Y + (1ll << 43)) >> 44);
    R = (__int128)(X - (u128)s * s);
    if (R < 0) { R += (__int128)(2 * s) - 1; s -= 1; }
    rem = (u128)R;
    return s;
}

// ---------------------------------------------------------------------------------------
// Correctly rounded hypot (Sect. 2).  With a = max(|x|,|y|), b = min:
//  * e_a - e_b >= (p+1)/2: b^2 < a ulp(a), so sqrt(a^2+b^2) lies strictly inside
//    (a, a + ulp(a)/2) and rounds to a;
//  * otherwise the exact sum of squares X is formed as an integer (a' = a scaled to
//    [1,2), units 2^-110 for double and 2^-52 for float; both subnormal: units of the
//    smallest subnormal squared) and the result is rounded from floor(sqrt X) (isqrt113,
//    isqrt55), the remainder and the truncated bits of b'^2, ties to even.  Neither version
//    uses a floating-point square root, and the double one no FP64 instruction, on this path.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double hypot_cr_body(double x, double y)
{
    uint64_t ab = dbits(x) & ~D_SIGN, bb = dbits(y) & ~D_SIGN;
    if (ab < bb) { uint64_t t = ab; ab = bb; bb = t; }
    if ((ab >> 52) == 0x7FF)                                 // inf, or a quiet nan
        return dfrom((ab << 12) ? (ab | 0x0008000000000000ull) : ab);
    if (bb == 0) return dfrom(ab);
    const int Ea = (int)(ab >> 52), Eb = (int)(bb >> 52);
    uint64_t A = ab & D_MANT, B = bb & D_MANT;
    int ea, eb;
    if (Ea) { A |= D_HID; ea = Ea - 1023; } else { int sh = __clzll((long long)A) - 11; A <<= sh; ea = -1022 - sh; }
    if (Eb) { B |= D_HID; eb = Eb - 1023; } else { int sh = __clzll((long long)B) - 11; B <<= sh; eb = -1022 - sh; }
    if (ea - eb >= 27) return dfrom(ab);
    u128 rem;
    if (Ea == 0) {
        // both subnormal: N = (a^2 + b^2) / q^2 with q = 2^-1074 (N < 2^105), the result
        // round(sqrt N) q; no ties (4N is even, (2k+1)^2 odd)
        const u128 N = (u128)ab * ab + (u128)bb * bb;
        const int k = (111 - (127 - clz128(N))) >> 1;               // N 4^k in [2^110, 2^113)
        uint64_t q = isqrt113(N << (2 * k), rem) >> k;              // floor(sqrt N)
        if (N - (u128)q * q > q) ++q;                               // sqrt N > q + 1/2
        return dfrom(q);                                            // q < 2^53
    }
    // exact a'^2 + b'^2 in units of 2^-110, with a sticky bit for truncated bits of b'^2
    u128 X = ((u128)A * A) << 6;
    const u128 B2 = (u128)B * B;
    const int sh = 2 * (eb - ea) + 6;
    bool sticky = false;
    if (sh >= 0) X += B2 << sh;
    else { const int k = -sh; sticky = (B2 << (128 - k)) != 0; X += B2 >> k; }
    // sqrt(X 2^-110) = sqrt(X) 2^-55 in [1, 2 sqrt 2): 53 bits of floor(sqrt X), round bit,
    // sticky from the lower bits, the remainder and the truncated b'^2
    const uint64_t s = isqrt113(X, rem);
    const int er = (s >> 56) ? 1 : 0;
    const int cut = 3 + er;
    uint64_t R = s >> cut;
    const bool rb = (s >> (cut - 1)) & 1;
    const bool st = (s & ((1ull << (cut - 1)) - 1)) != 0 || rem != 0 || sticky;
    int E = ea + er + 1023;
    if (rb && (st || (R & 1))) {
        ++R;
        if (R >> 53) { R >>= 1; ++E; }
    }
    if (E >= 2047) return dfrom(0x7FFull << 52);
    return dfrom(((uint64_t)E << 52) | (R & D_MANT));
}

static __device__ __noinline__ uint64_t hypot_cr_bits(uint64_t x, uint64_t y) { return dbits(hypot_cr_body(dfrom(x), dfrom(y))); }
__device__ __forceinline__ double hypot_cr(double x, double y) { return dfrom(hypot_cr_bits(dbits(x), dbits(y))); }

// floor(sqrt(X)) for an integer X in [2^52, 2^55), and the remainder, on the integer
// pipes: s0 from the FP32 reciprocal square root of X's leading 31 bits is within 2^6.1 of
// sqrt(X); one correction s + (X - s0^2) Y 2^-58 (Y = y 2^45 ~ 2^57 / sqrt(X), a 32-bit
// integer; the residual exact, its leading 31 bits times Y one 32x32->64-bit product) is
// within 1/2 + 2^-14 (quadratic term 2^-14.8, Y's error 2^-15.5, truncation 2^-23); the
// sign of X - s^2 then gives floor(sqrt X).
__device__ __forceinline__ uint32_t isqrt55(uint64_t X, uint64_t &rem)
{
    const float xf = __uint2float_rz((uint32_t)(X >> 24));           // [2^28, 2^31)
    const float y = rsqrtf(xf);                                       // 2^12 / sqrt(X)
    const int64_t Y = (int64_t)__float2uint_rn(y * 0x1p45f);
    uint64_t s = __float2uint_rn(xf * y * 4096.0f);
    int64_t R = (int64_t)(X - s * s);                                 // |R| < 2^34.7
    s += (uint64_t)(((int64_t)(int32_t)(R >> 4) * Y + (1ll << 53)) >> 54);
    R = (int64_t)(X - s * s);
    if (R < 0) { R += (int64_t)(2 * s) - 1; s -= 1; }
    rem = (uint64_t)R;
    return (uint32_t)s;
}

__device__ __forceinline__ float hypot_cr_body(float x, float y)
{
    uint32_t ab = fbits(x) & ~F_SIGN, bb = fbits(y) & ~F_SIGN;
    if (ab < bb) { uint32_t t = ab; ab = bb; bb = t; }
    if ((ab >> 23) == 0xFF)                                  // inf, or a quiet nan
        return ffrom((ab << 9) ? (ab | 0x00400000u) : ab);
    if (bb == 0) return ffrom(ab);
    const int Ea = (int)(ab >> 23), Eb = (int)(bb >> 23);
    uint32_t A = ab & F_MANT, B = bb & F_MANT;
    int ea, eb;
    if (Ea) { A |= F_HID; ea = Ea - 127; } else { int sh = __clz((int)A) - 8; A <<= sh; ea = -126 - sh; }
    if (Eb) { B |= F_HID; eb = Eb - 127; } else { int sh = __clz((int)B) - 8; B <<= sh; eb = -126 - sh; }
    if (ea - eb >= 13) return ffrom(ab);
    uint64_t rem;
    if (Ea == 0) {
        // both subnormal: N = (a^2 + b^2) / q^2, q = 2^-149 (N < 2^47), the result
        // round(sqrt N) q; no ties
        const uint64_t N = (uint64_t)ab * ab + (uint64_t)bb * bb;
        const int k = (53 - (63 - __clzll((long long)N))) >> 1;       // N 4^k in [2^52, 2^55)
        uint32_t q = isqrt55(N << (2 * k), rem) >> k;                 // floor(sqrt N)
        if (N - (uint64_t)q * q > q) ++q;
        return ffrom(q);                                            // q < 2^24
    }
    // exact a'^2 + b'^2 in units of 2^-52, with a sticky bit for truncated bits of b'^2
    uint64_t X = ((uint64_t)A * A) << 6;
    const uint64_t B2 = (uint64_t)B * B;
    const int sh = 2 * (eb - ea) + 6;
    bool sticky = false;
    if (sh >= 0) X += B2 << sh;
    else { const int k = -sh; sticky = (B2 << (64 - k)) != 0; X += B2 >> k; }
    const uint32_t s = isqrt55(X, rem);                             // sqrt(X) 2^-26 in [1, 2 sqrt 2)
    const int er = (s >> 27) ? 1 : 0;
    const int cut = 3 + er;
    uint32_t R = s >> cut;
    const bool rb = (s >> (cut - 1)) & 1;
    const bool st = (s & ((1u << (cut - 1)) - 1)) != 0 || rem != 0 || sticky;
    int E = ea + er + 127;
    if (rb && (st || (R & 1))) {
        ++R;
        if (R >> 24) { R >>= 1; ++E; }
    }
    if (E >= 255) return ffrom(0xFFu << 23);
    return ffrom(((uint32_t)E << 23) | (R & F_MANT));
}
static __device__ __noinline__ float hypot_cr(float x, float y) { return hypot_cr_body(x, y); }

// ---------------------------------------------------------------------------------------
// A hypot that is not correctly rounded, for Alg. 1's branch for that case: the scaled
// formula of LAPACK's xLAPY2, w sqrt(1 + (z/w)^2) with w = max(|x|,|y|), z = min(|x|,|y|),
// each step one IEEE rounding to nearest: q = z/w, r = fma(q, q, 1), w * sqrt(r).  The
// steps neither overflow nor underflow (q <= 1, 1 <= r <= 2); only the last product may
// overflow, to infinity.  Relative error below 3.5 u, u = 2^-p, to first order: the
// rounding of q changes sqrt(1 + q^2) by at most u, that of r by u/2, the root's and the
// product's by u each.  The quotient is the method's division; the square root is the
// FP64 (FP32) pipe's.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double hypot_ncr_body(double x, double y)
{
    double a = absv(x), b = absv(y);
    if (is_inf(a) || is_inf(b)) return dfrom(0x7FFull << 52);
    if (!is_fin(a) || !is_fin(b)) return dfrom(0x7FF8000000000000ull);
    if (pos_lt(a, b)) { const double t = a; a = b; b = t; }
    if (eq0(b)) return a;
    const double q = div_rn(b, a);
    return __dmul_rn(a, __dsqrt_rn(__fma_rn(q, q, 1.0)));
}
static __device__ __noinline__ uint64_t hypot_ncr_bits(uint64_t x, uint64_t y) { return dbits(hypot_ncr_body(dfrom(x), dfrom(y))); }
__device__ __forceinline__ double hypot_ncr(double x, double y) { return dfrom(hypot_ncr_bits(dbits(x), dbits(y))); }

__device__ __forceinline__ float hypot_ncr_body(float x, float y)
{
    float a = fabsf(x), b = fabsf(y);
    if (is_inf(a) || is_inf(b)) return ffrom(0xFFu << 23);
    if (!is_fin(a) || !is_fin(b)) return ffrom(0x7FC00000u);
    if (a < b) { const float t = a; a = b; b = t; }
    if (b == 0.0f) return a;
    const float q = __fdiv_rn(b, a);
    return __fmul_rn(a, __fsqrt_rn(__fmaf_rn(q, q, 1.0f)));
}
static __device__ __noinline__ float hypot_ncr(float x, float y) { return hypot_ncr_body(x, y); }

// ---------------------------------------------------------------------------------------
// eq. (EXT) for double: fl(FL(FL(x1 y1 +- x2 y2) / d)) with FL = IEEE binary128 rounding
// (113 bits, ties to even) and fl = binary64 rounding with gradual underflow, emulated
// exactly in integers.  The caller then divides by sec(theta) in double.  All operands
// are finite and non-zero; d > 0.
// ---------------------------------------------------------------------------------------
struct q113 { u128 m; int e; bool neg; };   // value (-1)^neg * m * 2^e

__device__ __forceinline__ void dmant(double x, uint64_t &M, int &e, bool &neg)
{
    uint64_t b = dbits(x);
    neg = (b >> 63) != 0;
    M = b & D_MANT;
    int E = (int)((b >> 52) & 0x7FF);
    if (E) { M |= D_HID; e = E - 1023 - 52; }
    else { int sh = __clzll((long long)M) - 11; M <<= sh; e = -1022 - sh - 52; }
}

// round the non-negative integer value m * 2^e (+ a sticky fraction below bit 0) to 113 bits
__device__ __forceinline__ void round113(u128 m, int e, bool sticky, u128 &M, int &E)
{
    int msb = 127 - clz128(m);
    if (msb > 112) {
        int k = msb - 112;
        bool rbit = (m >> (k - 1)) & 1;
        bool st = sticky || (k > 1 && (m << (129 - k)) != 0);
        M = m >> k;
        E = e + k;
        if (rbit && (st || (M & 1))) {
            M += 1;
            if ((M >> 113) != 0) { M >>= 1; E += 1; }
        }
    } else {
        M = m << (112 - msb);
        E = e - (112 - msb);
    }
}

__device__ __forceinline__ double ext_num_div_body(double x1, double y1, double x2, double y2, bool sub, double d)
{
    uint64_t a1, b1, a2, b2; int ea1, eb1, ea2, eb2; bool na1, nb1, na2, nb2;
    dmant(x1, a1, ea1, na1); dmant(y1, b1, eb1, nb1);
    dmant(x2, a2, ea2, na2); dmant(y2, b2, eb2, nb2);
    // exact products, normalised with the top bit at position 126
    u128 P1 = (u128)a1 * b1, P2 = (u128)a2 * b2;
    int s1 = clz128(P1) - 1, s2 = clz128(P2) - 1;
    P1 <<= s1; P2 <<= s2;
    int f1 = ea1 + eb1 - s1, f2 = ea2 + eb2 - s2;
    bool n1 = na1 ^ nb1, n2 = na2 ^ nb2 ^ sub;
    // larger magnitude first
    bool swap = (f2 > f1) || (f2 == f1 && P2 > P1);
    u128 L = swap ? P2 : P1, S = swap ? P1 : P2;
    int fL = swap ? f2 : f1, fS = swap ? f1 : f2;
    bool nL = swap ? n2 : n1, nS = swap ? n1 : n2;
    int dsh = fL - fS;
    bool sticky;
    u128 Sal;
    if (dsh == 0) { Sal = S; sticky = false; }
    else if (dsh >= 127) { Sal = 0; sticky = true; }
    else { Sal = S >> dsh; sticky = (S << (128 - dsh)) != 0; }
    u128 sum;
    if (nL == nS) sum = L + Sal;
    else sum = sticky ? (L - Sal - 1) : (L - Sal);
    if (sum == 0 && !sticky) return 0.0;                    // exact cancellation: +0
    u128 M1; int E1;
    round113(sum, fL, sticky, M1, E1);                     // FL(x1 y1 +- x2 y2)
    // FL(M1 2^E1 / d): integer quotient floor(M1 2^56 / Md), 116 or 117 bits, by 20-bit digits
    uint64_t Md; int ed; bool nd;
    dmant(d, Md, ed, nd);
    uint64_t r = (uint64_t)(M1 >> 61);                      // top 52 bits of M1, below Md
    u128 rest = (M1 & ((((u128)1) << 61) - 1)) << 56;      // the remaining 117 bits
    const float mhi = __uint2float_rn((uint32_t)(Md >> 29));  // exact, in [2^23, 2^24)
    u128 q = 0;
    int left = 117;
#pragma unroll 1
    while (left > 0) {
        int w = left >= 20 ? 20 : left;
        left -= w;
        u128 rp = ((u128)r << w) | ((rest >> left) & ((((u128)1) << w) - 1));
        float rhi = __uint2float_rn((uint32_t)(rp >> 49));   // exact: rp < 2^73
        float qf = __fmul_rn(__fdiv_rn(rhi, mhi), 1048576.0f);
        uint64_t qd = __float2uint_rz(qf);           // qf <= 2^21
        if (qd > (1ull << w)) qd = 1ull << w;
        u128 prod = (u128)qd * Md;
#pragma unroll 1
        while (prod > rp) { --qd; prod -= Md; }
        u128 rr = rp - prod;
#pragma unroll 1
        while (rr >= Md) { ++qd; rr -= Md; }
        r = (uint64_t)rr;
        q = (q << w) | qd;
    }
    // quotient value = (q + r/Md) 2^(E1 + 52 - ed_true - 56) with ed_true = ed + 52
    u128 M2; int E2;
    round113(q, E1 - 56 - ed, r != 0, M2, E2);
    // fl: round the 113-bit value M2 2^E2 (M2 in [2^112, 2^113)) to double
    int etrue = E2 + 112;
    bool neg = nL;
    if (etrue > 1023) return neg ? -__longlong_as_double(0x7FF0000000000000ll) : __longlong_as_double(0x7FF0000000000000ll);
    int k = (etrue >= -1022) ? 60 : (-1074 - E2);          // bits of M2 below the binary64 quantum
    if (k > 114) return neg ? -0.0 : 0.0;
    uint64_t Mr;
    if (k >= 113) {
        // M2 < 2^113 <= 2^k: the result is 0 or the smallest subnormal
        bool rbit = (k == 113);                             // bit k-1 = 112 is the leading 1
        bool st = M2 != (((u128)1) << 112);                 // bits below the leading one
        Mr = (rbit && st) ? 1 : 0;
    } else {
        bool rbit = (M2 >> (k - 1)) & 1;
        bool st = (k > 1) && ((M2 << (129 - k)) != 0);
        Mr = (uint64_t)(M2 >> k);
        if (rbit && (st || (Mr & 1))) Mr += 1;
    }
    uint64_t bits;
    if (etrue >= -1022) {
        int Eb = etrue + 1023;
        if ((Mr >> 53) != 0) { Mr >>= 1; Eb += 1; }
        if (Eb >= 2047) bits = 0x7FFull << 52;
        else bits = ((uint64_t)Eb << 52) | (Mr & D_MANT);
    } else {
        bits = Mr;                                          // subnormal (or 2^-1022 after a carry)
    }
    return dfrom(bits | (neg ? D_SIGN : 0));
}
static __device__ __noinline__ uint64_t ext_num_div_bits(uint64_t x1, uint64_t y1, uint64_t x2, uint64_t y2, bool sub, uint64_t d)
{
    return dbits(ext_num_div_body(dfrom(x1), dfrom(y1), dfrom(x2), dfrom(y2), sub, dfrom(d)));
}
__device__ __forceinline__ double ext_num_div(double x1, double y1, double x2, double y2, bool sub, double d)
{
    return dfrom(ext_num_div_bits(dbits(x1), dbits(y1), dbits(x2), dbits(y2), sub, dbits(d)));
}

// eq. (EXT) for float: the wide type is double, where the products of floats are exact
// eq. (EXT) for binary32 with binary64 as the wide type: the products are exact in binary64,
// the sum or difference and the quotient are rounded to binary64, then to binary32.  The
// quotient uses the FP64 divider: the binary32 kernel leaves the FP64 pipe mostly idle, so
// that is cheaper here than the integer-pipe division.
static __device__ __noinline__ float ext_num_div(float x1, float y1, float x2, float y2, bool sub, float d)
{
    double p2 = (double)x2 * (double)y2;
    double num = fma((double)x1, (double)y1, sub ? -p2 : p2);
    double q = num / (double)d;
    return __double2float_rn(q);
}

}  // namespace k2
