// Correctly rounded Taylor coefficients and step-N difference tables of one
// block (Sect. IV: R_t of degree d at the block's first argument X_t; Sect.
// IV-A hierarchical method), compiled for host and device.
//
//   c_k = RN(2^E_k f^(k)(X_t)/k!) mod 2^W,  E_k = W + log2(s) + k (e_in - p)
//
// with X_t = M 2^(e_in - p), M = 2^(p-1) + j_t.  exp and 2^x take one
// enclosure of f(X_t) at precision P = E_0 + guard for every order (E_0 is
// the largest scale); log takes one enclosure for k = 0 and exact rationals
// (-1)^(k-1) / (k X^k) for k >= 1.  A coefficient is accepted when both ends
// of its enclosure round alike; the caller retries undecided blocks with
// more limbs (Ziv's strategy).  RN rounds halves up (floor(v + 1/2)); halves
// only occur for exact values, which are handled exactly.
#pragma once

#include "fxp.cuh"

namespace tmd {

enum { COEFF_MAX_DEG = 4, COEFF_MAX_LIMBS = 3, LN2_LIMBS = 13, LN2_BITS = 768 };

// Constant inputs of the coefficient routine: reciprocals of small divisors
// and an enclosure of ln 2 with LN2_BITS fractional bits.
struct CoeffConsts {
    fx::DivTable div;
    fx::U<LN2_LIMBS> ln2_lo, ln2_hi;
};

struct CoeffJob {
    int func, e_in, p, d, L, scale_log2, log2_N;
};

namespace cf_detail {

// ln 2 enclosure at P <= LN2_BITS fractional bits into NL limbs
template <int NL>
TMD_HD void ln2_at(const CoeffConsts& C, unsigned P, fx::U<NL>& lo, fx::U<NL>& hi) {
    fx::U<LN2_LIMBS> a = C.ln2_lo, b = C.ln2_hi;
    const unsigned s = LN2_BITS - P;
    const bool up = fx::low_bits(b, s);
    fx::shr(a, s);
    fx::shr(b, s);
    if (up) fx::add_u64(b, 1);
    for (int i = 0; i < NL; i++) {
        lo.w[i] = i < LN2_LIMBS ? a.w[i] : 0;
        hi.w[i] = i < LN2_LIMBS ? b.w[i] : 0;
    }
}

// round x / 2^s to nearest (halves up), s >= 1
template <int NL>
TMD_HD void rn_shift(fx::U<NL>& x, unsigned s) {
    fx::U<NL> h;
    fx::set_pow2(h, s - 1);
    fx::add(x, h);
    fx::shr(x, s);
}

template <int NL>
TMD_HD void store_mod_w(const fx::U<NL>& x, bool neg, int L, uint64_t* out) {
    uint64_t c = 1;
    for (int l = 0; l < L; l++) {
        uint64_t w = x.w[l];
        if (neg) {
            w = ~w + c;
            c = (w == 0 && c) ? 1 : 0;
        }
        out[l] = w;
    }
}

// exact (-1)^(k-1) 2^sh / (k M^k) rounded to nearest, mod 2^W
template <int NL>
TMD_HD bool log_exact(uint64_t M, int k, int sh, const CoeffConsts& C, int L, uint64_t* out) {
    if (sh < 0 || sh + 2 >= 64 * NL) return false;
    const bool neg = (k % 2) == 0;
    fx::U<NL> den, x;
    fx::set_zero(den);
    den.w[0] = (uint64_t)k;
    for (int i = 0; i < k; i++)
        if (fx::mul_u64(den, M)) return false;
    fx::set_pow2(x, (unsigned)sh + 1);
    fx::add(x, den);
    if (neg) {
        fx::U<NL> one;
        fx::set_zero(one);
        one.w[0] = 1;
        fx::sub(x, one);
    }
    // floor((2 num + den [- 1]) / (2 den)) as a chain of exact floors
    fx::div_u64(x, C.div.r[2]);
    fx::div_u64(x, C.div.r[k]);
    const fx::Recip RM = fx::make_recip(M);
    for (int i = 0; i < k; i++) fx::div_u64(x, RM);
    store_mod_w(x, neg, L, out);
    return true;
}

}  // namespace cf_detail

// c[k*L + l] for k = 0..d.  Returns false when a rounding stays undecided
// at this width (retry with a wider NL) or a width is exceeded.
template <int NL>
TMD_HD bool block_coeffs(const CoeffJob& J, uint64_t M, int guard, const CoeffConsts& C, uint64_t* c) {
    using namespace fx;
    const int W = 64 * J.L;
    const int E0 = W + J.scale_log2;
    const unsigned P = (unsigned)((E0 > 0 ? E0 : 0) + guard);
    const unsigned q = (unsigned)(J.p - J.e_in);
    if ((int)P + 96 > 64 * NL) return false;
    const uint64_t fact[5] = {1, 1, 2, 6, 24};
    if (J.func == 2) {  // log
        Enc<NL> ln2, f;
        cf_detail::ln2_at<NL>(C, P, ln2.lo, ln2.hi);
        if (!log_enc<NL>(M, J.p, J.e_in, P, ln2, C.div, f)) return false;
        const int s = (int)P - E0;
        if (s < 1) return false;
        cf_detail::rn_shift(f.lo, (unsigned)s);
        cf_detail::rn_shift(f.hi, (unsigned)s);
        if (!equal(f.lo, f.hi)) return false;
        cf_detail::store_mod_w(f.lo, false, J.L, c);
        for (int k = 1; k <= J.d; k++) {
            const int Ek = E0 + k * (J.e_in - J.p);
            if (!cf_detail::log_exact<NL>(M, k, Ek + k * (int)q, C, J.L, c + k * J.L)) return false;
        }
        return true;
    }
    // exp or 2^x: one enclosure of f(X_t) with P2 >= P fractional bits
    const unsigned P2 = P + 16;
    Enc<NL> f;
    bool exact = false;
    if (J.func == 0) {
        if (!exp_small<NL>(M, q, P2, C.div, f)) return false;
    } else {
        if (q == 0 || (M & ((1ull << q) - 1)) == 0) {  // 2^X at an integer X
            set_pow2(f.lo, P2 + (unsigned)(q >= 64 ? 0 : (M >> q)));
            f.hi = f.lo;
            exact = true;
        } else {
            U<NL> llo, lhi;
            cf_detail::ln2_at<NL>(C, P2 + 16, llo, lhi);
            U<NL> ylo = llo, yhi = lhi;
            mul_u64(ylo, M);
            shr(ylo, q);
            mul_u64(yhi, M);
            const bool up = low_bits(yhi, q);
            shr(yhi, q);
            if (up) add_u64(yhi, 1);
            // the argument has P2 + 16 fractional bits; Xc bounds X ln 2 < 2^(e_in)
            const uint64_t Xc = (uint64_t)1 << (J.e_in > 0 ? J.e_in : 0);
            uint64_t e_lo, e_hi;
            U<NL> vlo, vhi;
            if (!exp_big<NL>(ylo, P2 + 16, Xc, C.div, vlo, e_lo)) return false;
            if (!exp_big<NL>(yhi, P2 + 16, Xc, C.div, vhi, e_hi)) return false;
            add_u64(vhi, e_hi);
            shr(vlo, 16);
            const bool up2 = low_bits(vhi, 16);
            shr(vhi, 16);
            if (up2) add_u64(vhi, 1);
            f.lo = vlo;
            f.hi = vhi;
        }
    }
    U<NL> l2lo, l2hi;
    if (J.func == 1) cf_detail::ln2_at<NL>(C, P2, l2lo, l2hi);
    U<NL> plo = f.lo, phi = f.hi;  // f (ln 2)^k enclosure, updated per order
    for (int k = 0; k <= J.d; k++) {
        if (J.func == 1 && k > 0) {
            U<NL> t;
            mul_shr(plo, l2lo, P2, t);
            plo = t;
            // upper end: ceil of the product
            U<NL> hprod;
            mul_shr(phi, l2hi, P2, hprod);
            add_u64(hprod, 1);
            phi = hprod;
            exact = false;
        }
        U<NL> lo = plo, hi = phi;
        if (k >= 2) {
            div_u64(lo, C.div.r[fact[k]]);
            const uint64_t rem = div_u64(hi, C.div.r[fact[k]]);
            if (rem) add_u64(hi, 1);
        }
        const int Ek = E0 + k * (J.e_in - J.p);
        const int s = (int)P2 - Ek;
        if (s < 1) return false;
        if (s >= 64 * NL) {
            // the scaled value is below 2^(Ek - P2 + bits) < 1/2: rounds to 0
            if (bit_length(hi) + 1 >= (unsigned)s) return false;
            for (int l = 0; l < J.L; l++) c[k * J.L + l] = 0;
            continue;
        }
        cf_detail::rn_shift(lo, (unsigned)s);
        cf_detail::rn_shift(hi, (unsigned)s);
        if (!equal(lo, hi)) return false;
        cf_detail::store_mod_w(lo, false, J.L, c + k * J.L);
    }
    (void)exact;
    return true;
}

// The 2d+1 table words from the coefficients: w = 0..d are Delta^w g0(0) with
// g0(i) = R(iN), w = d+1..2d are Delta^(w-d-1) g1(0) with
// g1(i) = R(iN+1) - R(iN), all mod 2^W.
TMD_HD void block_table_words(const CoeffJob& J, const uint64_t* c, uint64_t* table) {
    using namespace fx;
    const int L = J.L, d = J.d;
    const uint64_t N = 1ull << J.log2_N;
    U<COEFF_MAX_LIMBS> g0[COEFF_MAX_DEG + 1], g1[COEFF_MAX_DEG];
    for (int i = 0; i <= d; i++) {
        for (int pass = 0; pass < 2; pass++) {
            const uint64_t y = (uint64_t)i * N + (uint64_t)pass;
            U<COEFF_MAX_LIMBS> acc;
            set_zero(acc);
            for (int l = 0; l < L; l++) acc.w[l] = c[d * L + l];
            for (int k = d - 1; k >= 0; k--) {
                mul_u64(acc, y);
                U<COEFF_MAX_LIMBS> ck;
                set_zero(ck);
                for (int l = 0; l < L; l++) ck.w[l] = c[k * L + l];
                add(acc, ck);
                for (int l = L; l < COEFF_MAX_LIMBS; l++) acc.w[l] = 0;  // mod 2^W
            }
            if (pass == 0) {
                g0[i] = acc;
            } else if (i < d) {
                U<COEFF_MAX_LIMBS> t = acc;
                sub(t, g0[i]);
                for (int l = L; l < COEFF_MAX_LIMBS; l++) t.w[l] = 0;
                g1[i] = t;
            }
        }
    }
    for (int lev = 0; lev <= d; lev++) {
        for (int l = 0; l < L; l++) table[lev * L + l] = g0[0].w[l];
        for (int i = 0; i + lev < d; i++) {  // g0[i] <- g0[i+1] - g0[i]  (mod 2^W)
            U<COEFF_MAX_LIMBS> t = g0[i + 1];
            sub(t, g0[i]);
            for (int l = L; l < COEFF_MAX_LIMBS; l++) t.w[l] = 0;
            g0[i] = t;
        }
    }
    for (int lev = 0; lev < d; lev++) {
        for (int l = 0; l < L; l++) table[(d + 1 + lev) * L + l] = g1[0].w[l];
        for (int i = 0; i + lev + 1 < d; i++) {
            U<COEFF_MAX_LIMBS> t = g1[i + 1];
            sub(t, g1[i]);
            for (int l = L; l < COEFF_MAX_LIMBS; l++) t.w[l] = 0;
            g1[i] = t;
        }
    }
}

}  // namespace tmd
