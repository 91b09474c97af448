// Fixed-size multiword integers and rigorous enclosures of exp, 2^x and log
// for the correctly rounded Taylor coefficients of the block tables.
//
// Compiled for both host and device: the library's host path and its table
// kernel run this same code, so the CPU tests of the host path pin the
// arithmetic the GPU executes.
//
// A value v >= 0 is enclosed as lo / 2^P <= v <= hi / 2^P with lo, hi
// unsigned integers of NL 64-bit limbs (little-endian).  Series are summed
// with truncating arithmetic, and the accumulated truncation plus the tail of
// the series are bounded explicitly (same bounds as documented for each
// routine).  Divisions by 64-bit integers use the 2-by-1 division with a
// precomputed reciprocal of Moller and Granlund, "Improved division by
// invariant integers" (IEEE Trans. Computers, 2011), restated from its
// mathematics: for a normalised divisor d (top bit set) and
// v = floor((2^128 - 1)/d) - 2^64, the quotient of (u1 2^64 + u0) by d,
// u1 < d, is the high word of v u1 + (u1 2^64 + u0) plus one, corrected by at
// most two adjustments of the remainder.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define TMD_HD __host__ __device__ __forceinline__
#else
#define TMD_HD inline
#endif

namespace tmd {
namespace fx {

TMD_HD uint64_t mulhi(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

TMD_HD int clz64(uint64_t x) {  // x != 0
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return __builtin_clzll(x);
#endif
}

template <int NL>
struct U {
    uint64_t w[NL];
};

template <int NL>
TMD_HD void set_zero(U<NL>& a) {
#pragma unroll
    for (int i = 0; i < NL; i++) a.w[i] = 0;
}

template <int NL>
TMD_HD void set_pow2(U<NL>& a, unsigned e) {  // e < 64 NL
#pragma unroll
    for (int i = 0; i < NL; i++) a.w[i] = ((unsigned)i == e / 64) ? (1ull << (e % 64)) : 0ull;
}

template <int NL>
TMD_HD bool is_zero(const U<NL>& a) {
    uint64_t x = 0;
#pragma unroll
    for (int i = 0; i < NL; i++) x |= a.w[i];
    return x == 0;
}

template <int NL>
TMD_HD bool equal(const U<NL>& a, const U<NL>& b) {
    uint64_t x = 0;
#pragma unroll
    for (int i = 0; i < NL; i++) x |= a.w[i] ^ b.w[i];
    return x == 0;
}

// a += b, returns the carry out
template <int NL>
TMD_HD uint64_t add(U<NL>& a, const U<NL>& b) {
    uint64_t c = 0;
#pragma unroll
    for (int i = 0; i < NL; i++) {
        uint64_t s = a.w[i] + b.w[i];
        uint64_t c1 = s < a.w[i];
        uint64_t t = s + c;
        uint64_t c2 = t < s;
        a.w[i] = t;
        c = c1 | c2;
    }
    return c;
}

template <int NL>
TMD_HD uint64_t add_u64(U<NL>& a, uint64_t x) {
    uint64_t c = x;
#pragma unroll
    for (int i = 0; i < NL; i++) {
        uint64_t t = a.w[i] + c;
        c = t < c;
        a.w[i] = t;
    }
    return c;
}

// a -= b, returns the borrow out
template <int NL>
TMD_HD uint64_t sub(U<NL>& a, const U<NL>& b) {
    uint64_t br = 0;
#pragma unroll
    for (int i = 0; i < NL; i++) {
        uint64_t t = a.w[i] - b.w[i];
        uint64_t b1 = a.w[i] < b.w[i];
        uint64_t t2 = t - br;
        uint64_t b2 = t < br;
        a.w[i] = t2;
        br = b1 | b2;
    }
    return br;
}

// a *= m, returns the overflow limb
template <int NL>
TMD_HD uint64_t mul_u64(U<NL>& a, uint64_t m) {
    uint64_t c = 0;
#pragma unroll
    for (int i = 0; i < NL; i++) {
        uint64_t lo = a.w[i] * m;
        uint64_t hi = mulhi(a.w[i], m);
        uint64_t t = lo + c;
        hi += t < lo;
        a.w[i] = t;
        c = hi;
    }
    return c;
}

// out = in >> s for an NI-limb input into NL limbs, with static limb indices
// only (a runtime limb offset q is resolved by a compile-time-unrolled
// selection so that the limbs stay in registers on the device).
template <int NI, int NL>
TMD_HD void shift_down(const uint64_t* in, unsigned s, U<NL>& out) {
    const unsigned q = s / 64, r = s % 64;
#pragma unroll
    for (int i = 0; i < NL; i++) out.w[i] = 0;
#pragma unroll
    for (int qq = 0; qq < NI; qq++) {
        if ((unsigned)qq == q) {
#pragma unroll
            for (int i = 0; i < NL; i++) {
                const uint64_t lo = (i + qq < NI) ? in[i + qq] : 0;
                const uint64_t hi = (i + qq + 1 < NI) ? in[i + qq + 1] : 0;
                out.w[i] = r ? (lo >> r) | (hi << (64 - r)) : lo;
            }
        }
    }
}

// a >>= s
template <int NL>
TMD_HD void shr(U<NL>& a, unsigned s) {
    U<NL> t;
    shift_down<NL, NL>(a.w, s, t);
    a = t;
}

// a <<= s, bits shifted out are lost
template <int NL>
TMD_HD void shl(U<NL>& a, unsigned s) {
    const unsigned q = s / 64, r = s % 64;
    U<NL> t;
#pragma unroll
    for (int i = 0; i < NL; i++) t.w[i] = 0;
#pragma unroll
    for (int qq = 0; qq < NL; qq++) {
        if ((unsigned)qq == q) {
#pragma unroll
            for (int i = 0; i < NL; i++) {
                const uint64_t hi = (i - qq >= 0) ? a.w[i - qq] : 0;
                const uint64_t lo = (i - qq - 1 >= 0) ? a.w[i - qq - 1] : 0;
                t.w[i] = r ? (hi << r) | (lo >> (64 - r)) : hi;
            }
        }
    }
    a = t;
}

// true iff a has a set bit below position s
template <int NL>
TMD_HD bool low_bits(const U<NL>& a, unsigned s) {
    uint64_t x = 0;
#pragma unroll
    for (int i = 0; i < NL; i++) {
        const unsigned lo = 64u * (unsigned)i;
        if (lo + 64 <= s)
            x |= a.w[i];
        else if (lo < s)
            x |= a.w[i] & ((1ull << (s - lo)) - 1);
    }
    return x != 0;
}

// number of significant bits (0 for a = 0)
template <int NL>
TMD_HD unsigned bit_length(const U<NL>& a) {
    for (int i = NL - 1; i >= 0; i--)
        if (a.w[i]) return 64u * (unsigned)i + 64u - (unsigned)clz64(a.w[i]);
    return 0;
}

// r = (a * b) >> s, truncated to NL limbs (the full product has 2 NL limbs)
template <int NL>
TMD_HD void mul_shr(const U<NL>& a, const U<NL>& b, unsigned s, U<NL>& r) {
    uint64_t p[2 * NL];
#pragma unroll
    for (int i = 0; i < 2 * NL; i++) p[i] = 0;
#pragma unroll
    for (int i = 0; i < NL; i++) {
        uint64_t c = 0;
#pragma unroll
        for (int j = 0; j < NL; j++) {
            uint64_t lo = a.w[i] * b.w[j];
            uint64_t hi = mulhi(a.w[i], b.w[j]);
            uint64_t t = p[i + j] + lo;
            hi += t < lo;
            uint64_t t2 = t + c;
            hi += t2 < c;
            p[i + j] = t2;
            c = hi;
        }
        p[i + NL] = c;
    }
    shift_down<2 * NL, NL>(p, s, r);
}

// r = floor(a b / 2^PA) - e, e in {0, 1}, for PA = 64 (NL - 2) + 60 (the
// working precision of the table products): the partial products a_i b_j
// with i + j <= NL - 4 are not formed.  They all lie below
// 2^(64 (NL - 2)) each, so together below 2^(64 (NL - 2) + 6) < 2^PA, and
// dropping them lowers the quotient by at most one.  Needs a b < 2^(64 NL + PA).
template <int NL>
TMD_HD void mul_trunc(const U<NL>& a, const U<NL>& b, U<NL>& r) {
    constexpr int K0 = NL - 3;
    uint64_t p[2 * NL];
#pragma unroll
    for (int i = 0; i < 2 * NL; i++) p[i] = 0;
#pragma unroll
    for (int i = 0; i < NL; i++) {
        uint64_t c = 0;
#pragma unroll
        for (int j = 0; j < NL; j++) {
            if (i + j < K0) continue;
            uint64_t lo = a.w[i] * b.w[j];
            uint64_t hi = mulhi(a.w[i], b.w[j]);
            uint64_t t = p[i + j] + lo;
            hi += t < lo;
            uint64_t t2 = t + c;
            hi += t2 < c;
            p[i + j] = t2;
            c = hi;
        }
        p[i + NL] = c;
    }
#pragma unroll
    for (int k = 0; k < NL; k++) {
        const uint64_t lo = p[k + NL - 2], hi = (k + NL - 1 < 2 * NL) ? p[k + NL - 1] : 0;
        r.w[k] = (lo >> 60) | (hi << 4);
    }
}

// ------------------------------------------------ division by a 64-bit word
struct Recip {
    uint64_t dn;  // divisor shifted left until its top bit is set
    uint64_t v;   // floor((2^128 - 1) / dn) - 2^64
    unsigned sh;  // the shift
};

// v = floor((2^128 - 1) / dn) - 2^64 from a double-precision estimate and
// exact integer corrections.  x = fl(2^64 / fl(dn)) has relative error
// below 2^-52, so v0 = floor((x - 1) 2^64) is within 2^13 + 2 of v; from
// v0 - 2^14 (not above v) the remainder r = 2^128 - 1 - (2^64 + v0) dn is
// exact, non-negative and below 2^80; its quotient by dn, estimated in
// double precision less one (never above the exact one), and at most a few
// unit steps give v with 0 <= r < dn.
TMD_HD Recip make_recip(uint64_t d) {
    Recip R;
    R.sh = (unsigned)clz64(d);
    R.dn = d << R.sh;
    const uint64_t dn = R.dn;
    const double two64 = 18446744073709551616.0;
    const double x = two64 / (double)dn;  // in [1, 2]
    const double e = (x - 1.0) * two64;   // exact scaling; below 2^64 + 2^13
    uint64_t v = e >= 18446744073709549568.0 ? ~0ull : (uint64_t)e;  // 2^64 - 2^11
    v = v > 16384 ? v - 16384 : 0;
    // r = 2^128 - 1 - (2^64 + v) dn: the product's high word dn + hi(v dn)
    // stays below 2^64 since v is not above the exact quotient
    const uint64_t plo = v * dn, phi = mulhi(v, dn) + dn;
    uint64_t rl = ~plo, rh = ~phi;
    const double rd = (double)rh * two64 + (double)rl;
    uint64_t del = (uint64_t)(rd / (double)dn);
    del = del > 0 ? del - 1 : 0;
    const uint64_t dlo = del * dn, dhi = mulhi(del, dn);
    const uint64_t b = rl < dlo ? 1ull : 0ull;
    rl -= dlo;
    rh -= dhi + b;
    v += del;
#pragma unroll 1
    for (int it = 0; it < 8 && (rh != 0 || rl >= dn); it++) {
        rh -= rl < dn ? 1ull : 0ull;
        rl -= dn;
        v++;
    }
    R.v = v;
    return R;
}

// quotient of (u1 2^64 + u0) by R.dn (u1 < R.dn), remainder in r
TMD_HD uint64_t div_2by1(uint64_t u1, uint64_t u0, const Recip& R, uint64_t& r) {
    uint64_t q0 = R.v * u1;
    uint64_t q1 = mulhi(R.v, u1);
    uint64_t t = q0 + u0;
    q1 += u1 + (t < q0 ? 1ull : 0ull);
    q0 = t;
    q1 += 1;
    uint64_t rr = u0 - q1 * R.dn;
    if (rr > q0) {
        q1 -= 1;
        rr += R.dn;
    }
    if (rr >= R.dn) {
        q1 += 1;
        rr -= R.dn;
    }
    r = rr;
    return q1;
}

// a = floor(a / d), returns a mod d (R = make_recip(d))
template <int NL>
TMD_HD uint64_t div_u64(U<NL>& a, const Recip& R) {
    const unsigned s = R.sh;
    uint64_t r = s ? (a.w[NL - 1] >> (64 - s)) : 0;  // < 2^s <= dn
#pragma unroll
    for (int i = NL - 1; i >= 0; i--) {
        uint64_t digit = s ? (a.w[i] << s) | (i > 0 ? a.w[i - 1] >> (64 - s) : 0) : a.w[i];
        a.w[i] = div_2by1(r, digit, R, r);
    }
    return r >> s;
}

// --------------------------------------------------------------- enclosures
template <int NL>
struct Enc {
    U<NL> lo, hi;
};

// Reciprocals of the small divisors of the series (n = 1 .. SMALL_DIV_MAX).
enum { SMALL_DIV_MAX = 512 };

struct DivTable {
    Recip r[SMALL_DIV_MAX + 1];
};

// exp(X) for X = y / 2^Q with y < 2^64 (one limb), P fractional bits:
// t_0 = 2^P, t_n = floor(t_{n-1} y / (2^Q n)); the truncation error of t_n
// satisfies e_n <= e_{n-1} X / n + 1, tracked with Xc = ceil(X); once
// t_n = 0 and n >= 2 Xc + 2 the true term is at most e_n and the tail after
// it at most the term.  Needs 64 NL >= P + bits(y) + bits(e^X) + 2.  When
// X < 1 and Q <= 64, y / 2^Q is applied as the one-limb multiplier
// y 2^(64-Q) followed by dropping the low limb (the same floor).
template <int NL>
TMD_HD bool exp_small(uint64_t y, unsigned Q, unsigned P, const DivTable& T, Enc<NL>& out) {
    const uint64_t Xc = Q >= 64 ? (y ? 1 : 0) : ((y >> Q) + ((y & ((1ull << Q) - 1)) ? 1 : 0));
    const bool fold = Q >= 1 && (Q == 64 || (Q < 64 && (y >> Q) == 0));
    const uint64_t yf = Q == 64 ? y : (fold ? y << (64 - Q) : 0);
    U<NL> t, S;
    set_pow2(t, P);
    S = t;
    uint64_t e = 0, E = 0;
    for (uint64_t n = 1; n <= SMALL_DIV_MAX; n++) {
        if (fold) {
            const uint64_t top = mul_u64(t, yf);
#pragma unroll
            for (int i = 0; i + 1 < NL; i++) t.w[i] = t.w[i + 1];
            t.w[NL - 1] = top;
        } else {
            mul_u64(t, y);
            shr(t, Q);
        }
        div_u64(t, T.r[n]);
        U<1> en;
        en.w[0] = e * Xc + n - 1;
        div_u64(en, T.r[n]);
        e = en.w[0] + 1;
        add(S, t);
        E += e;
        if (n >= 2 * Xc + 2 && is_zero(t)) {
            E += e + 1;
            out.lo = S;
            out.hi = S;
            add_u64(out.hi, E);
            return true;
        }
    }
    return false;
}

// exp(Y) for Y = y / 2^P given as an NL-limb fixed-point number (same bounds,
// with the product t y formed exactly and truncated once).
template <int NL>
TMD_HD bool exp_big(const U<NL>& y, unsigned P, uint64_t Xc, const DivTable& T, U<NL>& lo,
                    uint64_t& err) {
    U<NL> t, S, tmp;
    set_pow2(t, P);
    S = t;
    uint64_t e = 0, E = 0;
    for (uint64_t n = 1; n <= SMALL_DIV_MAX; n++) {
        mul_shr(t, y, P, tmp);
        t = tmp;
        div_u64(t, T.r[n]);
        e = (e * Xc + n - 1) / n + 1;
        add(S, t);
        E += e;
        if (n >= 2 * Xc + 2 && is_zero(t)) {
            E += e + 1;
            lo = S;
            err = E;
            return true;
        }
    }
    return false;
}

// ln 2 = sum_k 2 / ((2k+1) 3^(2k+1)): w_0 = floor(2^(P+1)/3),
// w_k = floor(w_{k-1}/9) (error <= 2), term = floor(w_k/(2k+1)) (error <= 2).
template <int NL>
TMD_HD bool ln2_enc(unsigned P, const DivTable& T, Enc<NL>& out) {
    U<NL> w, S;
    set_pow2(w, P + 1);
    div_u64(w, T.r[3]);
    S = w;
    uint64_t E = 1;
    for (uint64_t k = 1; 2 * k + 1 <= SMALL_DIV_MAX; k++) {
        div_u64(w, T.r[9]);
        U<NL> t = w;
        div_u64(t, T.r[2 * k + 1]);
        add(S, t);
        E += 2;
        if (is_zero(t)) {
            E += 1;
            out.lo = S;
            out.hi = S;
            add_u64(out.hi, E);
            return true;
        }
    }
    return false;
}

// atanh(num/den) for 0 <= num < den / 3 (den < 2^62), P fractional bits:
// S <= 2^P atanh(num/den) <= S + E.  w_0 = floor(2^P num/den) (error <= 1),
// w_k = w_{k-1} z^2 by two truncating multiply-divides (error <= 3),
// term_k = floor(w_k/(2k+1)) (error <= 2); the tail after a zero term is
// below 1.
template <int NL>
TMD_HD bool atanh_ratio(uint64_t num, uint64_t den, unsigned P, const DivTable& T, U<NL>& S, uint64_t& E) {
    const Recip Rd = make_recip(den);
    U<NL> w;
    set_pow2(w, P);
    mul_u64(w, num);
    div_u64(w, Rd);
    S = w;
    E = 1;
    for (uint64_t k = 1; 2 * k + 1 <= SMALL_DIV_MAX; k++) {
        mul_u64(w, num);
        div_u64(w, Rd);
        mul_u64(w, num);
        div_u64(w, Rd);
        U<NL> t = w;
        div_u64(t, T.r[2 * k + 1]);
        add(S, t);
        E += 2;
        if (is_zero(t)) {
            E += 1;
            return true;
        }
    }
    return false;
}

// log X for X = M 2^(e_in - p), 2^(p-1) <= M < 2^p, e_in >= 1:
// log X = e_in ln 2 - 2 atanh(z), z = (2^p - M)/(2^p + M) in (0, 1/3].
template <int NL>
TMD_HD bool log_enc(uint64_t M, int p, int e_in, unsigned P, const Enc<NL>& ln2, const DivTable& T,
                    Enc<NL>& out) {
    U<NL> S;
    uint64_t E;
    if (!atanh_ratio<NL>((1ull << p) - M, (1ull << p) + M, P, T, S, E)) return false;
    U<NL> two_hi = S, two_lo = S;
    add_u64(two_hi, E);
    mul_u64(two_hi, 2);
    mul_u64(two_lo, 2);
    out.lo = ln2.lo;
    mul_u64(out.lo, (uint64_t)e_in);
    out.hi = ln2.hi;
    mul_u64(out.hi, (uint64_t)e_in);
    if (sub(out.lo, two_hi)) return false;  // log X > 0 on the supported binades
    sub(out.hi, two_lo);
    return true;
}

}  // namespace fx
}  // namespace tmd
