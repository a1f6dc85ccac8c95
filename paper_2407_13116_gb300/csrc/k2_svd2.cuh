// One 2x2 SVD by the enhanced Kogbetliantz method (arXiv 2407.13116, Sect. 3), as a device
// function: one matrix per thread, everything in registers.
//
// Phases (Sect. 3): (1) zero-pattern type t and scale type from eq. (ts), prescaling by
// eqs. (eG), (s); (2) the simple cases of Sect. 3.1 or the URV of Sect. 3.2 (error-free for
// t' ~ 13, fully pivoted with eq. (QR15)/(EXT) for t' = 15); (3) the SVD of R by Alg. 1 and
// Alg. 2 after the transpose-swap of eq. (RT), the assembly of U and V (eqs. (UV15), (UV))
// with the left-vector heuristic of eqs. (p+t), (p-t), (tan+-), and the backscaling.
//
// Readings of the text (each also stated where it is used):
//  * class-9 types (0,1,2,4,6,8,9) are not scaled: s = 0 (Sect. 3.1, first sentence);
//  * ties in magnitude comparisons never swap (strict "<");
//  * sign(+-0) = +1; outputs -0 are returned as +0;
//  * eq. (EXT) is used for the element with the essential subtraction only when tan(theta)
//    is inexact, detected by fma(tan theta, g11''', -g21''') != 0 (Thm. 3.5);
//  * P~ of eq. (RT) is the anti-identity (the printed identity is a typesetting error);
//  * V = V_+ V-check P_sigma and U = S1 P_U S22 U(phi +- theta) S2 P_sigma (eq. (UV) with
//    V_+ of eq. (UV15));
//  * (cos, sin) of phi +- theta follow the direction of (D, N) with N, D the numerator and
//    denominator of eq. (tan+-); a zero D or an overflowing N/D gives (0, sign N); the bold
//    phi with an infinite tangent (tan psi = 0 after the swap) gives pi/2 +- theta exactly.
// With NCR = true (a separate variant) Alg. 1 takes its branch for a hypot that is not
// correctly rounded, and every hypot of the method is xLAPY2's scaled formula (hypot_ncr).
#pragma once
#include "k2_fp.cuh"

namespace k2 {

enum : int {
    FL_EXT = 0x01, FL_FALLBACK = 0x02, FL_SWAP = 0x04, FL_T2F2 = 0x08,
    FL_T2F3 = 0x10, FL_T2INF = 0x20, FL_TPINF = 0x40, FL_PSIG = 0x80,
    FL_T2NCR = 0x400
};

// class of each zero-pattern type, eq. (ts): 9, 3, 5, 13 or 15
__device__ __forceinline__ int cls_of(int t)
{
    // bit k of these masks marks the types of a class
    const unsigned c3 = (1u << 3) | (1u << 12), c5 = (1u << 5) | (1u << 10);
    const unsigned c13 = (1u << 7) | (1u << 11) | (1u << 13) | (1u << 14);
    unsigned b = 1u << t;
    return (t == 15) ? 15 : (b & c13) ? 13 : (b & c3) ? 3 : (b & c5) ? 5 : 9;
}

template <typename T> struct m22 { T a11, a21, a12, a22; };   // column-major 2x2

template <typename T> __device__ __forceinline__ void swap_rows(m22<T> &m)
{
    T t = m.a11; m.a11 = m.a21; m.a21 = t;
    t = m.a12; m.a12 = m.a22; m.a22 = t;
}
template <typename T> __device__ __forceinline__ void swap_cols(m22<T> &m)
{
    T t = m.a11; m.a11 = m.a12; m.a12 = t;
    t = m.a21; m.a21 = m.a22; m.a22 = t;
}
// IEEE negation (a sign-bit flip) on the integer pipes
__device__ __forceinline__ double ngt(double x) { return dfrom(dbits(x) ^ D_SIGN); }
__device__ __forceinline__ float ngt(float x) { return -x; }
template <typename T> __device__ __forceinline__ void neg_row(m22<T> &m, int r)
{
    if (r == 0) { m.a11 = ngt(m.a11); m.a12 = ngt(m.a12); } else { m.a21 = ngt(m.a21); m.a22 = ngt(m.a22); }
}
template <typename T> __device__ __forceinline__ void neg_col(m22<T> &m, int c)
{
    if (c == 0) { m.a11 = ngt(m.a11); m.a21 = ngt(m.a21); } else { m.a12 = ngt(m.a12); m.a22 = ngt(m.a22); }
}
template <typename T> __device__ __forceinline__ m22<T> rot(T c, T s)     // [[c,-s],[s,c]]
{
    m22<T> m; m.a11 = c; m.a21 = s; m.a12 = ngt(s); m.a22 = c; return m;
}
template <typename T> __device__ __forceinline__ m22<T> ident()
{
    m22<T> m; m.a11 = T(1); m.a21 = T(0); m.a12 = T(0); m.a22 = T(1); return m;
}

template <typename T> struct svd2_out {
    m22<T> U, V;
    ef<T> s1, s2;        // backscaled singular values, sigma1 >= sigma2
    int info;
};

// The method's hypot: correctly rounded (the paper's choice), or with NCR the scaled formula
// that is not, the case for which Alg. 1 has its own branch.
template <bool NCR, typename T> __device__ __forceinline__ T hyp(T x, T y)
{
    if (NCR) return hypot_ncr(x, y);
    return hypot_cr(x, y);
}

// sec = hypot(tan,1), cos = 1/sec, sin = tan/sec (Cor. 2.3, Lemma 3.2)
template <bool NCR = false, typename T> __device__ __forceinline__ void cos_sin(T tn, T &c, T &s)
{
    T sec = hyp<NCR>(tn, T(1));
    c = qdiv(T(1), sec);
    s = qdiv(tn, sec);
}

// Sect. 3.1, class 9: U = P_U diag(sign a, sign b), V = P_V, sigma' = (|a|, |b|)
template <typename T>
__device__ __forceinline__ void simple9(int tt, T g11, T g21, T g12, T g22, m22<T> &U, m22<T> &V, T &d1, T &d2)
{
    bool pu = false, pv = false;
    T a = T(0), b = T(0);
    switch (tt) {
    case 1: a = g11; break;
    case 2: pu = true; a = g21; break;
    case 4: pv = true; a = g12; break;
    case 8: pu = true; pv = true; a = g22; break;
    case 9:
        if (abs_lt(g11, g22)) { pu = pv = true; a = g22; b = g11; } else { a = g11; b = g22; }
        break;
    case 6:
        if (abs_lt(g12, g21)) { pu = true; a = g21; b = g12; } else { pv = true; a = g12; b = g21; }
        break;
    default: break;
    }
    U = ident<T>();
    if (pu) swap_rows(U);
    if (lt0(a)) neg_col(U, 0);
    if (lt0(b)) neg_col(U, 1);
    V = ident<T>();
    if (pv) swap_rows(V);
    d1 = absv(a); d2 = absv(b);
}

// Sect. 3.1, classes 3 (one non-zero column) and 5 (one non-zero row): one Givens rotation
template <typename T, bool NCR = false>
__device__ __forceinline__ void simple35(int tt, T g11, T g21, T g12, T g22, m22<T> &U, m22<T> &V, T &d1)
{
    bool col = (tt == 3 || tt == 12);
    bool p0;
    T x0, x1;
    if (col) { p0 = (tt == 12); x0 = p0 ? g12 : g11; x1 = p0 ? g22 : g21; }
    else { p0 = (tt == 10); x0 = p0 ? g21 : g11; x1 = p0 ? g22 : g12; }
    bool n0 = lt0(x0), n1 = lt0(x1);
    T y0 = absv(x0), y1 = absv(x1);
    bool p1 = pos_lt(y0, y1);
    T x = p1 ? y1 : y0, y = p1 ? y0 : y1;
    T c, s;
    cos_sin<NCR>(qdiv(y, x), c, s);
    d1 = hyp<NCR>(x, y);
    m22<T> R = rot(c, s);            // U_theta (column case) or V_theta (row case)
    if (p1) swap_rows(R);
    if (n0) neg_row(R, 0);
    if (n1) neg_row(R, 1);
    m22<T> P = ident<T>();
    if (p0) swap_rows(P);
    if (col) { U = R; V = P; } else { U = P; V = R; }
}

// State of the SVD of R~ (Sect. 3.3.1)
template <typename T> struct tri_out {
    bool swap, psig;
    T tanphi, cphi, sphi, tanpsi, cpsi, spsi;
    ef<T> s1, s2;
};

// Alg. 1's test fl(x / y) < eps (eps = 2^-p) for x, y > 0 given as (e,f) pairs, decided exactly
// without the division.  With d = e_x - e_y and f_x, f_y in [1, 2) on the grid 2^-(p-1), the
// quotient is q = (f_x / f_y) 2^d with f_x / f_y in (1/2, 2), and fl(q) < 2^-p exactly when q
// lies below the midpoint 2^-p (1 - 2^-(p+1)) between 2^-p and its predecessor (at the midpoint
// the tie goes to the even 2^-p):
//   * d < -p: q <= (2 - 2^-(p-1)) 2^-(p+1) = 2^-p (1 - 2^-p), below the midpoint;
//   * d > -p: q > 2^-p;
//   * d = -p: q >= 2^-p when f_x >= f_y; when f_x < f_y, f_x <= f_y - 2^-(p-1), so
//     f_x / f_y < 1 - 2^-p, below the midpoint.
template <typename T> __device__ __forceinline__ bool quot_below_eps(ef<T> x, ef<T> y)
{
    const int d = x.e - y.e;
    return d < -fpt<T>::P || (d == -fpt<T>::P && pos_lt(x.f, y.f));
}

// The cos/sin divisions of the triangular SVD: on the FP64 divider when FDIV (the caller's
// FP64 pipe has room: general matrices), else as every other division.  Same results.
// (double: the out-of-line fdiv_rn, one copy of the divide sequence for every call site;
// 2^27 wide-range matrices 32.0 ms against 32.2 with the sequence inline at each site)
template <bool FDIV> __device__ __forceinline__ double csdiv(double a, double b) { return FDIV ? fdiv_rn(a, b) : qdiv(a, b); }
template <bool FDIV> __device__ __forceinline__ float csdiv(float a, float b) { return FDIV ? a / b : qdiv(a, b); }

// Alg. 1 and Alg. 2 on R = [[r11, r12], [0, r22]] (all > 0), with the transpose-swap of eq. (RT).
// NCR: the hypot that is not correctly rounded, and Alg. 1's branch for it.
template <typename T, bool FDIV = false, bool NCR = false>
__device__ __forceinline__ void tri_svd(T r11, T r12, T r22, tri_out<T> &z, int &flags)
{
    z.swap = pos_lt(r11, r22);
    T ra = z.swap ? r22 : r11, rb = r12, rc = z.swap ? r11 : r22;
    if (z.swap) flags |= FL_SWAP;
    ef<T> era = ef_of(ra), erb = ef_of(rb), erc = ef_of(rc);
    T t2;
    bool t2inf = false;
    // The cases of Alg. 1 only choose the operands of one division: the plain quotient
    // 2 r~22 / r~12 of eq. (t2f''), or the (e,f) quotient (2 r~12 r~22) / Y of eqs. (t2f''')
    // and (t2f') with Y = r~11^2 or (h - r~22)(h + r~22).  One call site, so that a warp
    // whose lanes take different cases divides once.
    int kind = -1;                                         // 0: plain; 1: (e,f); 2: t2 = inf
    ef<T> Y;
    Y.e = 0; Y.f = T(1);
    if (pos_eq(ra, rc)) {                                        // eq. (t2f'')
        kind = 0;
        flags |= FL_T2F2;
    } else if (pos_eq(rb, rc)) {                                 // eq. (t2f''')
        kind = 1; Y = ef_mul(era, era);
        flags |= FL_T2F3;
    } else if (quot_below_eps(era, erb)) {                       // eq. (t2f''), only for t' ~ 13
        kind = 0;
        flags |= FL_T2F2;
    } else if (!NCR) {                                     // eq. (t2f')
        T h = hypot_cr(ra, rb);
        if (pos_eq(h, rc)) kind = 2;
        else { kind = 1; Y = ef_mul(ef_minus(h, rc), ef_plus(h, rc)); }
    }
    if (kind >= 0) {
        if (kind == 2) { t2 = T(0); t2inf = true; }
        else {
            const ef<T> X = ef_mul(ef_pow2(1, erb), erc);
            const T q = qdiv(kind == 0 ? T(2) * rc : X.f, kind == 0 ? rb : Y.f);
            if (kind == 0) t2 = q;
            else { ef<T> w; renorm(q, X.e - Y.e, w.e, w.f); t2 = ef_fl(w); }
        }
    } else {                                               // NCR: Alg. 1 without squaring
        T x, y, num;
        if (pos_lt(rb, ra)) { x = qdiv(rb, ra); y = qdiv(rc, ra); num = (T(2) * x) * y; }
        else { x = qdiv(ra, rb); y = qdiv(rc, rb); num = T(2) * y; }
        T den = fma(x - y, x + y, T(1));
        if (!gt0(den)) den = T(0);                         // max(den, 0), -0 -> +0
        t2 = qdiv(num, den);
        flags |= FL_T2NCR;
    }
    if (is_inf(t2)) t2inf = true;
    T tf;
    if (t2inf) { tf = T(1); flags |= FL_T2INF; }
    else tf = qdiv(t2, T(1) + hyp<NCR>(t2, T(1)));           // eq. (tf)
    T secf = hyp<NCR>(tf, T(1));
    z.tanphi = tf;
    z.cphi = csdiv<FDIV>(T(1), secf);
    z.sphi = csdiv<FDIV>(tf, secf);
    // Alg. 2
    T t = fma(rc, tf, rb);                                 // eq. (tp)
    T tp = qdiv(t, ra);
    ef<T> s1, s2;
    if (is_inf(tp)) {                                       // eqs. (tp'), (s'')
        ef<T> et = ef_of(t);
        ef<T> ecos = ef_div(era, et);
        z.cpsi = ef_fl(ecos);
        z.spsi = T(1);
        s1 = et;
        s2 = ef_mul(erc, ecos);
        flags |= FL_TPINF;
    } else {                                               // eq. (s')
        T secp = hyp<NCR>(tp, T(1));
        z.cpsi = csdiv<FDIV>(T(1), secp);
        z.spsi = csdiv<FDIV>(tp, secp);
        ef<T> sf = ef_div(ef_of(secf), ef_of(secp));
        s1 = ef_div(era, sf);
        s2 = ef_mul(erc, sf);
    }
    z.tanpsi = tp;
    z.psig = ef_prec(s1, s2);                              // eq. (prec)
    if (z.psig) { z.s1 = s2; z.s2 = s1; flags |= FL_PSIG; }
    else { z.s1 = s1; z.s2 = s2; }
}

// U-check = P~ V_psi (swap) or U_phi, then P_sigma; V-check = P~ U_phi (swap) or V_psi, then P_sigma
template <typename T> __device__ __forceinline__ m22<T> ucheck(const tri_out<T> &z)
{
    m22<T> m;
    if (z.swap) { m.a11 = z.spsi; m.a21 = z.cpsi; m.a12 = z.cpsi; m.a22 = ngt(z.spsi); }
    else m = rot(z.cphi, z.sphi);
    if (z.psig) swap_cols(m);
    return m;
}
template <typename T> __device__ __forceinline__ m22<T> vcheck(const tri_out<T> &z)
{
    m22<T> m;
    if (z.swap) { m.a11 = z.sphi; m.a21 = z.cphi; m.a12 = z.cphi; m.a22 = ngt(z.sphi); }
    else m = rot(z.cpsi, z.spsi);
    if (z.psig) swap_cols(m);
    return m;
}

// eq. (QR15) with Thm. 3.5: r12 and r22 by fma, except the one with the essential
// subtraction (r22 when g12''' and g22''' have equal signs, else r12), which comes from eq.
// (EXT) when tan(theta) is inexact (Lemma 3.4); both divided by sec(theta).  Written with a
// single call of each primitive, so that a warp whose lanes take different cases runs the
// long eq. (EXT) body once, not once per case.  FDIV: see csdiv.
template <typename T, bool FDIV>
__device__ __forceinline__ void urv15_r(T g11, T g21, T g12, T g22, T tth, T secth, T &r12, T &r22, int &flags)
{
    T n12 = fma(g22, tth, g12);
    T n22 = fma(ngt(g12), tth, g22);
    if (!eq0(fma(tth, g11, ngt(g21)))) {                 // tan(theta) inexact: Thm. 3.5
        const bool e22 = lt0(g12) == lt0(g22);
        const T e = ext_num_div(e22 ? g22 : g12, g11, e22 ? g12 : g22, g21, e22, g11);
        if (e22) n22 = e; else n12 = e;
        flags |= FL_EXT;
    }
    r12 = csdiv<FDIV>(n12, secth);
    r22 = csdiv<FDIV>(n22, secth);
}

// Phase 1 (Sect. 3.1, eqs. (eG), (s)): the type t of G, the prescaling exponent
// s = e_nu - e_G - (scale type + extra) (class 9 is not scaled: s = 0), G <- 2^s G (exact
// for s >= 0, one rounding per element otherwise), and the type t' of the scaled matrix.
// extra = 0 in the method; the standalone entry allows more headroom.
template <typename T>
__device__ __forceinline__ void phase1(T &g11, T &g21, T &g12, T &g22, int extra, int &t, int &s, int &tp)
{
    t = !eq0(g11) | (!eq0(g21) << 1) | (!eq0(g12) << 2) | (!eq0(g22) << 3);
    const int cls = cls_of(t);
    s = 0;
    if (cls != 9) {
        int eG = INT_MIN;
        if (!eq0(g11)) eG = max(eG, fpt<T>::expo(g11));
        if (!eq0(g21)) eG = max(eG, fpt<T>::expo(g21));
        if (!eq0(g12)) eG = max(eG, fpt<T>::expo(g12));
        if (!eq0(g22)) eG = max(eG, fpt<T>::expo(g22));
        s = fpt<T>::ENU - eG - (cls == 15 ? 2 : 1) - extra;
        g11 = fpt<T>::scale(g11, s); g21 = fpt<T>::scale(g21, s);
        g12 = fpt<T>::scale(g12, s); g22 = fpt<T>::scale(g22, s);
    }
    tp = !eq0(g11) | (!eq0(g21) << 1) | (!eq0(g12) << 2) | (!eq0(g22) << 3);
}

// What phase 3 (Sect. 3.3) needs from phases 1 and 2: R and the transformations already
// applied.  Class 13: R = [[r11, r12], [0, r22]] after the permutations P_U, P_V and the
// signs S11 (na), S12, S22 of Sect. 3.2.1.  Class 15: R' after S12 and S22, with tan and
// sec of theta (eq. (QR15)), P_U, P_V and the row signs S1 (na, nb) of Sect. 3.2.2.
template <typename T> struct svd2_mid {
    T r11, r12, r22, tth, secth;
    int s, t, tp, flags;
    bool c15, pu, pv, na, nb, n12, n22;
};

// Phases 1 and 2 (Sect. 3.1, 3.2).  Returns false when o is complete (the simple classes,
// the fallback of Sect. 3.2.2), true when phase 3 (svd2_b) must finish from m.  FDIV: the
// quotients r12, r22 of eq. (QR15) on the FP64 divider, FDIV_T: tan theta (see csdiv).
template <typename T, bool NCR = false, bool FDIV = false, bool FDIV_T = FDIV>
__device__ __forceinline__ bool svd2_a(T g11, T g21, T g12, T g22, svd2_out<T> &o, svd2_mid<T> &m)
{
    int t, s, tp, flags = 0;
    phase1(g11, g21, g12, g22, 0, t, s, tp);
    const int clsp = cls_of(tp);
    m.s = s; m.t = t; m.tp = tp;
    T d1 = T(0), d2 = T(0);

    if (clsp == 9) {
        simple9(tp, g11, g21, g12, g22, o.U, o.V, d1, d2);
    } else if (clsp == 3 || clsp == 5) {
        simple35<T, NCR>(tp, g11, g21, g12, g22, o.U, o.V, d1);
    } else if (clsp == 13) {
        // Sect. 3.2.1: permute to upper triangular, signs of row 1, column 2, row 2
        m.pu = (tp == 11 || tp == 14); m.pv = (tp == 7 || tp == 11);
        T a, b, d;
        if (tp == 7) { a = g12; b = g11; d = g21; }
        else if (tp == 11) { a = g22; b = g21; d = g11; }
        else if (tp == 14) { a = g21; b = g22; d = g12; }
        else { a = g11; b = g12; d = g22; }
        m.na = lt0(a); a = absv(a); if (m.na) b = ngt(b);
        m.n12 = lt0(b); b = absv(b); if (m.n12) d = ngt(d);
        m.n22 = lt0(d); d = absv(d);
        m.r11 = a; m.r12 = b; m.r22 = d;
        m.c15 = false; m.nb = false; m.flags = flags;
        return true;
    } else {
        // Sect. 3.2.2: fully pivoted URV of a matrix without zeros
        T w1 = hyp<NCR>(g11, g21), w2 = hyp<NCR>(g12, g22);
        const bool pv = pos_lt(w1, w2);
        if (pv) { T x = g11; g11 = g12; g12 = x; x = g21; g21 = g22; g22 = x; w1 = w2; }
        const bool n1a = lt0(g11), n1b = lt0(g21);            // S1
        if (n1a) { g11 = ngt(g11); g12 = ngt(g12); }
        if (n1b) { g21 = ngt(g21); g22 = ngt(g22); }
        const bool pu = pos_lt(g11, g21);
        if (pu) { T x = g11; g11 = g21; g21 = x; x = g12; g12 = g22; g22 = x; }
        // eq. (QR15)
        // tan(theta): the phase's only integer-pipe division, inlined (2^27 wide-range
        // matrices: 31.1 ms against 32.0 through the shared out-of-line body)
        const T tth = FDIV_T ? csdiv<FDIV_T>(g21, g11) : qdiv_inl(g21, g11);
        const T secth = hyp<NCR>(tth, T(1));
        T r11 = w1, r12, r22;
        urv15_r<T, FDIV>(g11, g21, g12, g22, tth, secth, r12, r22, flags);
        if (eq0(r12) || eq0(r22)) {
            // R'' of type 9 (or 1) or 5: finish as Sect. 3.1, G' = S1 P_U U_theta R'' P_V^T
            flags |= FL_FALLBACK;
            const T cth = qdiv(T(1), secth), sth = qdiv(tth, secth);
            m22<T> Ur, Vr;
            if (eq0(r12)) {
                simple9<T>(!eq0(r22) ? 9 : 1, r11, T(0), T(0), r22, Ur, Vr, d1, d2);
            } else {
                simple35<T, NCR>(5, r11, T(0), r12, T(0), Ur, Vr, d1);
                d2 = T(0);
            }
            // U_theta Ur, with Ur a signed permutation: pick and negate columns of U_theta
            m22<T> M;
            bool c0first = !eq0(Ur.a11);                 // non-zero of column 0 in row 0
            T sg0 = c0first ? Ur.a11 : Ur.a21, sg1 = c0first ? Ur.a22 : Ur.a12;
            T u0a = c0first ? cth : ngt(sth), u0b = c0first ? sth : cth;   // U_theta column k0
            T u1a = c0first ? ngt(sth) : cth, u1b = c0first ? cth : sth;   // U_theta column k1
            M.a11 = lt0(sg0) ? ngt(u0a) : u0a; M.a21 = lt0(sg0) ? ngt(u0b) : u0b;
            M.a12 = lt0(sg1) ? ngt(u1a) : u1a; M.a22 = lt0(sg1) ? ngt(u1b) : u1b;
            if (pu) swap_rows(M);
            if (n1a) neg_row(M, 0);
            if (n1b) neg_row(M, 1);
            o.U = M;
            if (pv) swap_rows(Vr);
            o.V = Vr;
        } else {
            m.n12 = lt0(r12);
            if (m.n12) { r12 = ngt(r12); r22 = ngt(r22); }        // R'' S12
            m.n22 = lt0(r22);
            if (m.n22) r22 = ngt(r22);                         // S22 R'
            m.r11 = r11; m.r12 = r12; m.r22 = r22; m.tth = tth; m.secth = secth;
            m.c15 = true; m.pu = pu; m.pv = pv; m.na = n1a; m.nb = n1b; m.flags = flags;
            return true;
        }
    }
    o.s1 = ef_pow2(-s, ef_of(d1));                         // Sect. 3.3.2: 2^-s (.) sigma~'
    o.s2 = ef_pow2(-s, ef_of(d2));
    o.info = t | (tp << 4) | (flags << 8);
    return false;
}

// Phase 3 (Sect. 3.3) from the state of svd2_a: the SVD of R by Alg. 1 and Alg. 2, the
// assembly of U and V (class 15 with the heuristic of eqs. (p+t), (p-t), (tan+-), (UV)),
// and the backscaling.  FDIV: see csdiv.
template <typename T, bool FDIV = false, bool NCR = false>
__device__ __forceinline__ void svd2_b(const svd2_mid<T> &m, svd2_out<T> &o)
{
    int flags = m.flags;
    tri_out<T> z;
    tri_svd<T, FDIV, NCR>(m.r11, m.r12, m.r22, z, flags);
    m22<T> V = vcheck(z);                                  // V = P_V S12 V-check
    if (m.n12) neg_row(V, 1);
    if (m.pv) swap_rows(V);
    o.V = V;
    if (!m.c15) {
        m22<T> U = ucheck(z);                              // U = P_U S11 S22 U-check
        if (m.na) neg_row(U, 0);
        if (m.n22) neg_row(U, 1);
        if (m.pu) swap_rows(U);
        o.U = U;
    } else {
        // U = S1 P_U S22 U(phi +- theta) S2 P_sigma: eqs. (p+t), (p-t), (tan+-), (UV)
        const T tth = m.tth, secth = m.secth;
        const bool plus = !m.n22;
        const T tb = z.swap ? qdiv(T(1), z.tanpsi) : z.tanphi;
        T ca, sa;
        if (is_inf(tb)) {
            const T cth = qdiv(T(1), secth), sth = qdiv(tth, secth);
            ca = plus ? ngt(sth) : sth; sa = cth;
        } else {
            const T N = plus ? tb + tth : tb - tth;
            const T D = plus ? fma(ngt(tb), tth, T(1)) : fma(tb, tth, T(1));
            if (eq0(D)) { ca = T(0); sa = lt0(N) ? T(-1) : T(1); }
            else {
                const T ta = qdiv(N, D);
                if (is_inf(ta)) { ca = T(0); sa = lt0(N) ? T(-1) : T(1); }
                else {
                    T c0, s0;
                    cos_sin<NCR>(ta, c0, s0);
                    if (lt0(D)) { ca = ngt(c0); sa = ngt(s0); } else { ca = c0; sa = s0; }
                }
            }
        }
        m22<T> U = rot(ca, sa);
        if (z.swap) neg_col(U, 1);                         // S2
        if (m.n22) neg_row(U, 1);                          // S22
        if (m.pu) swap_rows(U);                            // P_U
        if (m.na) neg_row(U, 0);                           // S1
        if (m.nb) neg_row(U, 1);
        if (z.psig) swap_cols(U);                          // P_sigma
        o.U = U;
    }
    o.s1 = ef_pow2(-m.s, z.s1);                            // Sect. 3.3.2: 2^-s (.) sigma~'
    o.s2 = ef_pow2(-m.s, z.s2);
    o.info = m.t | (m.tp << 4) | (flags << 8);
}

// FDIV: see csdiv; the results do not depend on it.  NCR: see tri_svd.
template <typename T, bool FDIV = false, bool NCR = false>
__device__ __forceinline__ void svd2(T g11, T g21, T g12, T g22, svd2_out<T> &o)
{
    int t, s, tp, flags = 0;
    phase1(g11, g21, g12, g22, 0, t, s, tp);
    const int clsp = cls_of(tp);
    bool simple = true;
    T d1 = T(0), d2 = T(0);

    if (clsp == 9) {
        simple9(tp, g11, g21, g12, g22, o.U, o.V, d1, d2);
    } else if (clsp == 3 || clsp == 5) {
        simple35<T, NCR>(tp, g11, g21, g12, g22, o.U, o.V, d1);
    } else if (clsp == 13) {
        // Sect. 3.2.1: permute to upper triangular, signs of row 1, column 2, row 2
        simple = false;
        bool pu = (tp == 11 || tp == 14), pv = (tp == 7 || tp == 11);
        T a, b, d;
        if (tp == 7) { a = g12; b = g11; d = g21; }
        else if (tp == 11) { a = g22; b = g21; d = g11; }
        else if (tp == 14) { a = g21; b = g22; d = g12; }
        else { a = g11; b = g12; d = g22; }
        bool n11 = lt0(a); a = absv(a); if (n11) b = ngt(b);
        bool n12 = lt0(b); b = absv(b); if (n12) d = ngt(d);
        bool n22 = lt0(d); d = absv(d);
        tri_out<T> z;
        tri_svd<T, FDIV, NCR>(a, b, d, z, flags);
        m22<T> U = ucheck(z);                              // U = P_U S11 S22 U-check
        if (n11) neg_row(U, 0);
        if (n22) neg_row(U, 1);
        if (pu) swap_rows(U);
        m22<T> V = vcheck(z);                              // V = P_V S12 V-check
        if (n12) neg_row(V, 1);
        if (pv) swap_rows(V);
        o.U = U; o.V = V; o.s1 = z.s1; o.s2 = z.s2;
    } else {
        // Sect. 3.2.2: fully pivoted URV of a matrix without zeros
        T w1 = hyp<NCR>(g11, g21), w2 = hyp<NCR>(g12, g22);
        bool pv = pos_lt(w1, w2);
        if (pv) { T x = g11; g11 = g12; g12 = x; x = g21; g21 = g22; g22 = x; w1 = w2; }
        bool n1a = lt0(g11), n1b = lt0(g21);            // S1
        if (n1a) { g11 = ngt(g11); g12 = ngt(g12); }
        if (n1b) { g21 = ngt(g21); g22 = ngt(g22); }
        bool pu = pos_lt(g11, g21);
        if (pu) { T x = g11; g11 = g21; g21 = x; x = g12; g12 = g22; g22 = x; }
        // eq. (QR15)
        const T tth = qdiv(g21, g11);
        const T secth = hyp<NCR>(tth, T(1));
        T r11 = w1, r12, r22;
        urv15_r<T, false>(g11, g21, g12, g22, tth, secth, r12, r22, flags);
        if (eq0(r12) || eq0(r22)) {
            // R'' of type 9 (or 1) or 5: finish as Sect. 3.1, G' = S1 P_U U_theta R'' P_V^T
            flags |= FL_FALLBACK;
            const T cth = qdiv(T(1), secth), sth = qdiv(tth, secth);
            m22<T> Ur, Vr;
            if (eq0(r12)) {
                simple9<T>(!eq0(r22) ? 9 : 1, r11, T(0), T(0), r22, Ur, Vr, d1, d2);
            } else {
                simple35<T, NCR>(5, r11, T(0), r12, T(0), Ur, Vr, d1);
                d2 = T(0);
            }
            // U_theta Ur, with Ur a signed permutation: pick and negate columns of U_theta
            m22<T> M;
            bool c0first = !eq0(Ur.a11);                 // non-zero of column 0 in row 0
            T sg0 = c0first ? Ur.a11 : Ur.a21, sg1 = c0first ? Ur.a22 : Ur.a12;
            T u0a = c0first ? cth : ngt(sth), u0b = c0first ? sth : cth;   // U_theta column k0
            T u1a = c0first ? ngt(sth) : cth, u1b = c0first ? cth : sth;   // U_theta column k1
            M.a11 = lt0(sg0) ? ngt(u0a) : u0a; M.a21 = lt0(sg0) ? ngt(u0b) : u0b;
            M.a12 = lt0(sg1) ? ngt(u1a) : u1a; M.a22 = lt0(sg1) ? ngt(u1b) : u1b;
            if (pu) swap_rows(M);
            if (n1a) neg_row(M, 0);
            if (n1b) neg_row(M, 1);
            o.U = M;
            if (pv) swap_rows(Vr);
            o.V = Vr;
        } else {
            simple = false;
            bool n12 = lt0(r12);
            if (n12) { r12 = ngt(r12); r22 = ngt(r22); }            // R'' S12
            bool n22 = lt0(r22);
            if (n22) r22 = ngt(r22);                           // S22 R'
            tri_out<T> z;
            tri_svd<T, FDIV, NCR>(r11, r12, r22, z, flags);
            m22<T> V = vcheck(z);                          // V = P_V S12 V-check
            if (n12) neg_row(V, 1);
            if (pv) swap_rows(V);
            o.V = V;
            // U = S1 P_U S22 U(phi +- theta) S2 P_sigma: eqs. (p+t), (p-t), (tan+-), (UV)
            const bool plus = !n22;
            const T tb = z.swap ? qdiv(T(1), z.tanpsi) : z.tanphi;
            T ca, sa;
            if (is_inf(tb)) {
                const T cth = qdiv(T(1), secth), sth = qdiv(tth, secth);
                ca = plus ? ngt(sth) : sth; sa = cth;
            } else {
                const T N = plus ? tb + tth : tb - tth;
                const T D = plus ? fma(ngt(tb), tth, T(1)) : fma(tb, tth, T(1));
                if (eq0(D)) { ca = T(0); sa = lt0(N) ? T(-1) : T(1); }
                else {
                    const T ta = qdiv(N, D);
                    if (is_inf(ta)) { ca = T(0); sa = lt0(N) ? T(-1) : T(1); }
                    else {
                        T c0, s0;
                        cos_sin<NCR>(ta, c0, s0);
                        if (lt0(D)) { ca = ngt(c0); sa = ngt(s0); } else { ca = c0; sa = s0; }
                    }
                }
            }
            m22<T> U = rot(ca, sa);
            if (z.swap) neg_col(U, 1);                    // S2
            if (n22) neg_row(U, 1);                        // S22
            if (pu) swap_rows(U);                          // P_U
            if (n1a) neg_row(U, 0);                        // S1
            if (n1b) neg_row(U, 1);
            if (z.psig) swap_cols(U);                      // P_sigma
            o.U = U;
            o.s1 = z.s1; o.s2 = z.s2;
        }
    }
    if (simple) { o.s1 = ef_of(d1); o.s2 = ef_of(d2); }
    o.s1 = ef_pow2(-s, o.s1);                              // Sect. 3.3.2: 2^-s (.) sigma~'
    o.s2 = ef_pow2(-s, o.s2);
    o.info = t | (tp << 4) | (flags << 8);
}

}  // namespace k2
