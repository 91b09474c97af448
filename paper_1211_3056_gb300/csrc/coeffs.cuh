// Correctly rounded Taylor coefficients and step-N difference tables of one
// block (Sect. IV: R_t of degree d at the block's first argument X_t; Sect.
// IV-A hierarchical method), compiled for host and device.
//
//   c_k = RN(2^E_k f^(k)(X_t)/k!) mod 2^W,  E_k = W + log2(s) + k (e_in - p)
//
// with X_t = M 2^(e_in - p), M = 2^(p-1) + j_t.  exp and 2^x take one
// enclosure of f(X_t) at precision P = E_0 + guard for every order (E_0 is
// the largest scale); log takes one enclosure for k = 0 and exact rationals
// (-1)^(k-1) / (k X^k) for k >= 1.  Above the binade [2, 4) exp and 2^x are
// range-reduced by the block's output exponent: with red = e_out - 1,
// f(X) = 2^red g(X), g(X) = exp(X - red ln 2) or 2^(X - red), in [1, 2), and
// 2^E_k f = 2^(E_k + red) g, so that the fixed-point widths are those of the
// binade [1, 2) whatever the size of f.  A coefficient is accepted when both ends
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
    int red;  // range-reduction exponent (0: none), see reduction_exponent
};

// red = e_out - 1 for exp and 2^x above the binade [2, 4), else 0 (the
// arguments of the smaller binades keep their direct evaluation).
TMD_HD int reduction_exponent(int func, int e_in, int e_out) { return (func != 2 && e_in > 2) ? e_out - 1 : 0; }

// X = M 2^-q is an integer (any shift q: for q >= 64, 0 <= X < 1 since
// M < 2^64, so only M = 0 is)
TMD_HD bool integer_arg(uint64_t M, unsigned q) {
    if (q >= 64) return M == 0;
    return (M & ((1ull << q) - 1)) == 0;
}

// ceil(M 2^-q) for M > 0, any shift q
TMD_HD uint64_t ceil_arg(uint64_t M, unsigned q) {
    if (q >= 64) return M ? 1 : 0;
    return (M >> q) + (integer_arg(M, q) ? 0 : 1);
}

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

// 2^X for X = M 2^-q (M not a multiple of 2^q) with PB fractional bits:
// exp of the outward-rounded argument X ln 2 with PB + 16 bits, both ends.
template <int NL>
TMD_HD bool exp2_arg(const CoeffJob& J, uint64_t M, unsigned PB, const CoeffConsts& C, fx::Enc<NL>& f) {
    using namespace fx;
    const unsigned q = (unsigned)(J.p - J.e_in);
    U<NL> llo, lhi;
    cf_detail::ln2_at<NL>(C, PB + 16, llo, lhi);
    U<NL> ylo = llo, yhi = lhi;
    mul_u64(ylo, M);
    shr(ylo, q);
    mul_u64(yhi, M);
    const bool up = low_bits(yhi, q);
    shr(yhi, q);
    if (up) add_u64(yhi, 1);
    // Xc = ceil(M 2^-q) bounds the argument X ln 2 < X
    const uint64_t Xc = ceil_arg(M, q);
    uint64_t e_lo, e_hi;
    U<NL> vlo, vhi;
    if (!exp_big<NL>(ylo, PB + 16, Xc, C.div, vlo, e_lo)) return false;
    if (!exp_big<NL>(yhi, PB + 16, Xc, C.div, vhi, e_hi)) return false;
    add_u64(vhi, e_hi);
    shr(vlo, 16);
    const bool up2 = low_bits(vhi, 16);
    shr(vhi, 16);
    if (up2) add_u64(vhi, 1);
    f.lo = vlo;
    f.hi = vhi;
    return true;
}

// exp(X) 2^-red = exp(r), r = X - red ln 2 in [0, ln 2), X = M 2^-q, with
// PB fractional bits.  r is enclosed from an enclosure of ln 2 with PB + 28
// fractional bits (red < 2^11, so red ln 2 is known to 2^-(PB+17)) and
// rounded outward to PB + 16 bits; exp is increasing, so exp(r_lo) and
// exp(r_hi) enclose exp(r).  False when the enclosure of r is not inside
// [0, 1) (red is not the output exponent's) or a width is exceeded.
template <int NL>
TMD_HD bool exp_reduced(const CoeffJob& J, uint64_t M, unsigned PB, const CoeffConsts& C, fx::Enc<NL>& f) {
    using namespace fx;
    const unsigned q = (unsigned)(J.p - J.e_in);
    const unsigned PA = PB + 28;
    if (J.red <= 0 || J.red >= 2048 || PA > LN2_BITS || PA < q || PA - q + 64 > 64u * NL) return false;
    U<NL> llo, lhi;
    cf_detail::ln2_at<NL>(C, PA, llo, lhi);
    mul_u64(llo, (uint64_t)J.red);
    mul_u64(lhi, (uint64_t)J.red);
    U<NL> rlo, rhi;
    set_zero(rlo);
    rlo.w[0] = M;
    shl(rlo, PA - q);
    rhi = rlo;
    if (sub(rlo, lhi)) return false;
    if (sub(rhi, llo)) return false;
    shr(rlo, 12);
    const bool up = low_bits(rhi, 12);
    shr(rhi, 12);
    if (up) add_u64(rhi, 1);
    if (bit_length(rhi) > PB + 16) return false;  // r < 1
    uint64_t e_lo, e_hi;
    U<NL> vlo, vhi;
    if (!exp_big<NL>(rlo, PB + 16, 1, C.div, vlo, e_lo)) return false;
    if (!exp_big<NL>(rhi, PB + 16, 1, C.div, vhi, e_hi)) return false;
    add_u64(vhi, e_hi);
    shr(vlo, 16);
    const bool up2 = low_bits(vhi, 16);
    shr(vhi, 16);
    if (up2) add_u64(vhi, 1);
    f.lo = vlo;
    f.hi = vhi;
    return true;
}

// Per-job anchor: an enclosure of f at the job's first block X_a (exp and
// 2^x: f(X_a) with P2 fractional bits; log: log X_a with P), at the
// precision of the job's first segment (the largest scale of the job).
// Blocks then evaluate only the short series of the offset X_t - X_a:
//   exp(X_t) = exp(X_a) exp(d),  2^X_t = 2^X_a exp(d ln 2),
//   log X_t = log X_a + 2 atanh((M_t - M_a)/(M_t + M_a)),
// with d = (M_t - M_a) 2^(e_in - p) small.
enum { ANCHOR_LIMBS = 8 };
struct Anchor {
    uint64_t Ma;
    uint32_t P;     // fractional bits of lo, hi
    uint32_t ok;
    int32_t red;    // the reduction exponent the anchor's value carries
    uint32_t pad;
    uint64_t lo[ANCHOR_LIMBS], hi[ANCHOR_LIMBS];
};

namespace cf_detail {

// fractional bits of the base enclosure of f for a block with this scale
TMD_HD unsigned base_bits(const CoeffJob& J, int guard) {
    const int E0 = 64 * J.L + J.scale_log2 + J.red;
    const unsigned P = (unsigned)((E0 > 0 ? E0 : 0) + guard);
    return J.func == 2 ? P : P + 16;
}

// direct enclosure of f(X) 2^-red (exp, 2^x: P2 = P + 16 bits; log: P bits)
template <int NL>
TMD_HD bool f_direct(const CoeffJob& J, uint64_t M, unsigned PB, const CoeffConsts& C, fx::Enc<NL>& f, bool& exact) {
    using namespace fx;
    const unsigned q = (unsigned)(J.p - J.e_in);
    exact = false;
    if (J.func == 2) {
        Enc<NL> ln2;
        ln2_at<NL>(C, PB, ln2.lo, ln2.hi);
        return log_enc<NL>(M, J.p, J.e_in, PB, ln2, C.div, f);
    }
    if (J.func == 0) return J.red ? exp_reduced<NL>(J, M, PB, C, f) : exp_small<NL>(M, q, PB, C.div, f);
    if (J.red) {  // 2^(X - red), X - red = (M - red 2^q) 2^-q in [0, 1)
        if (q == 0 || q >= 64 || (M >> q) != (uint64_t)J.red) return false;
        M -= (uint64_t)J.red << q;
    }
    if (integer_arg(M, q)) {  // 2^X at an integer X (then q < 64 or X = 0)
        set_pow2(f.lo, PB + (unsigned)(q >= 64 ? 0 : (M >> q)));
        f.hi = f.lo;
        exact = true;
        return true;
    }
    return exp2_arg<NL>(J, M, PB, C, f);
}

}  // namespace cf_detail

template <int NL>
TMD_HD bool job_anchor(const CoeffJob& J0, uint64_t Ma, int guard, const CoeffConsts& C, Anchor& A) {
    static_assert(NL == ANCHOR_LIMBS, "anchors are stored with ANCHOR_LIMBS limbs");
    A.Ma = Ma;
    A.P = cf_detail::base_bits(J0, guard);
    A.ok = 0;
    A.red = J0.red;
    A.pad = 0;
    if ((int)A.P + 80 > 64 * NL) return false;
    fx::Enc<NL> f;
    bool exact;
    if (!cf_detail::f_direct<NL>(J0, Ma, A.P, C, f, exact)) return false;
    for (int i = 0; i < NL; i++) {
        A.lo[i] = f.lo.w[i];
        A.hi[i] = f.hi.w[i];
    }
    A.ok = 1;
    return true;
}

namespace cf_detail {

// enclosure of f(X_t) with PB fractional bits from the anchor (false when
// the anchor does not apply; the anchor's own block is evaluated directly)
template <int NL>
TMD_HD bool f_anchored(const CoeffJob& J, uint64_t M, unsigned PB, const CoeffConsts& C, const Anchor& A,
                       fx::Enc<NL>& f) {
    using namespace fx;
    // one reduction exponent: a reduced anchor serves the blocks of its
    // own output binade (there X_t - X_a < ln 2, or < 1 for 2^x)
    if (!A.ok || M <= A.Ma || A.P < PB || A.red != J.red) return false;
    Enc<NL> a;
    for (int i = 0; i < NL; i++) {
        a.lo.w[i] = i < ANCHOR_LIMBS ? A.lo[i] : 0;
        a.hi.w[i] = i < ANCHOR_LIMBS ? A.hi[i] : 0;
    }
    const unsigned sh = A.P - PB;
    if (sh) {
        const bool up = low_bits(a.hi, sh);
        shr(a.lo, sh);
        shr(a.hi, sh);
        if (up) add_u64(a.hi, 1);
    }
    const uint64_t dM = M - A.Ma;
    const unsigned q = (unsigned)(J.p - J.e_in);
    if (J.func == 2) {  // log X_t = log X_a + 2 atanh(dM / (M + Ma))
        U<NL> S;
        uint64_t E;
        if (!atanh_ratio<NL>(dM, M + A.Ma, PB, C.div, S, E)) return false;
        U<NL> two_lo = S, two_hi = S;
        add_u64(two_hi, E);
        mul_u64(two_lo, 2);
        mul_u64(two_hi, 2);
        f.lo = a.lo;
        f.hi = a.hi;
        add(f.lo, two_lo);
        add(f.hi, two_hi);
        return true;
    }
    Enc<NL> e;  // exp(d) or exp(d ln 2)
    if (J.func == 0) {
        if (!exp_small<NL>(dM, q, PB, C.div, e)) return false;
    } else {
        const CoeffJob Jd = J;
        if (!exp2_arg<NL>(Jd, dM, PB, C, e)) return false;
    }
    mul_shr(a.lo, e.lo, PB, f.lo);
    mul_shr(a.hi, e.hi, PB, f.hi);
    add_u64(f.hi, 1);
    return true;
}

}  // namespace cf_detail

// c[k*L + l] for k = 0..d.  Returns false when a rounding stays undecided
// at this width (retry with a wider NL) or a width is exceeded.  With an
// anchor of the block's job, f(X_t) comes from the anchored short series.
template <int NL>
TMD_HD bool block_coeffs(const CoeffJob& J, uint64_t M, int guard, const CoeffConsts& C, uint64_t* c,
                         const Anchor* anchor = nullptr) {
    using namespace fx;
    const int W = 64 * J.L;
    const int E0 = W + J.scale_log2 + J.red;  // f(X_t) is enclosed as 2^red g
    const unsigned P = (unsigned)((E0 > 0 ? E0 : 0) + guard);
    const unsigned q = (unsigned)(J.p - J.e_in);
    if ((int)P + 96 > 64 * NL) return false;
    const uint64_t fact[5] = {1, 1, 2, 6, 24};
    const unsigned PB = cf_detail::base_bits(J, guard);
    Enc<NL> f;
    bool exact = false;
    const bool integer_x = J.func == 1 && integer_arg(M, q);
    if (!(anchor && !integer_x && cf_detail::f_anchored<NL>(J, M, PB, C, *anchor, f)))
        if (!cf_detail::f_direct<NL>(J, M, PB, C, f, exact)) return false;
    if (J.func == 2) {  // log
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
    // exp or 2^x: the enclosure of f(X_t) has P2 = PB fractional bits
    const unsigned P2 = PB;
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
