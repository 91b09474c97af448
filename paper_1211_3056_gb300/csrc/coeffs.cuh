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

// the low L limbs of x (or of -x) into out[0 .. L), out[L .. COEFF_MAX_LIMBS)
// zeroed: every slot is written with a constant index, so that an array of
// coefficients in registers stays there
template <int NL>
TMD_HD void store_mod_w(const fx::U<NL>& x, bool neg, int L, uint64_t* out) {
    uint64_t c = 1;
#pragma unroll
    for (int l = 0; l < COEFF_MAX_LIMBS; l++) {
        uint64_t w = l < NL ? x.w[l < NL ? l : 0] : 0;
        if (neg) {
            w = ~w + c;
            c = (w == 0 && c) ? 1 : 0;
        }
        out[l] = l < L ? w : 0;
    }
}

// c_k = (-1)^(k-1) 2^sh / (k M^k) rounded to nearest, mod 2^W, for k = 1..d
// (halves rounded up for odd k and toward zero for even k), the slots above
// d zeroed; with step > 1 only the orders k = part (mod step).  One chain
// of exact floors serves every order (floor(floor(a/b) / c) =
// floor(a/(bc))): y_k = floor(2^(sh+1) / M^k), F = floor(y_k / k) =
// floor(2^(sh+1) / (k M^k)); the rounded value is F/2 for even F and
// (F+1)/2 for odd F, less one at a tie (the division exact) for even k.
template <int NL>
TMD_HD bool log_orders(uint64_t M, int d, int sh, const CoeffConsts& C, int L, uint64_t* c, int part = 0,
                       int step = 1) {
    if (sh < 0 || sh + 2 >= 64 * NL) return false;
    const fx::Recip RM = fx::make_recip(M);
    fx::U<NL> y;
    fx::set_pow2(y, (unsigned)sh + 1);
    bool exact = true;
    int have = 0;  // y = floor(2^(sh+1) / M^have)
#pragma unroll 1
    for (int k = part == 0 ? step : part; k <= COEFF_MAX_DEG; k += step) {
        if (k > d) {
#pragma unroll
            for (int l = 0; l < COEFF_MAX_LIMBS; l++) c[k * COEFF_MAX_LIMBS + l] = 0;
            continue;
        }
#pragma unroll 1
        while (have < k) {
            const uint64_t ry = fx::div_u64(y, RM);
            exact = exact && ry == 0;
            have++;
        }
        fx::U<NL> F = y;
        const uint64_t rk = fx::div_u64(F, C.div.r[k]);
        const bool neg = (k % 2) == 0;
        const bool up = (F.w[0] & 1) && !(neg && exact && rk == 0);
        fx::shr(F, 1);
        if (up) fx::add_u64(F, 1);
        store_mod_w(F, neg, L, c + k * COEFF_MAX_LIMBS);
    }
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

// Tables of the device path for exp, 2^x and log: entry (base, level i, b) is
// an enclosure of base^(b 2^(-8 i)), i = 1..10, b < 256 (base 0: e, base 1:
// 2), level 0 of base e holds e^n, n < 4, level 0 of "base" 2 holds
// log(256 + b) and its level 1 log(1 + b 2^-16); lo and hi ends of CT_LIMBS
// limbs with CT_BITS fractional bits.  An argument X = n + sum_i b_i
// 2^(-8 i) with at most 80 fractional bits then has e^X (2^X) as the product
// of at most 11 entries (2^n exact), with no series per block (the
// table-driven method of Tang's exponential, here with rigorous enclosures
// at every step); log X takes the entries of the argument's top 9 bits and
// of the next 8 and a short atanh series of the rest.
enum { CT_BASES = 3, CT_LEVELS = 11, CT_ENTRIES = 256, CT_LIMBS = 12, CT_BITS = 64 * CT_LIMBS - 68 };

TMD_HD size_t ct_index(int base, int level, int b, int end) {
    return ((((size_t)base * CT_LEVELS + (size_t)level) * CT_ENTRIES + (size_t)b) * 2 + (size_t)end) * CT_LIMBS;
}

constexpr size_t CT_WORDS = (size_t)CT_BASES * CT_LEVELS * CT_ENTRIES * 2 * CT_LIMBS;

// Entry (base, level, b) of the tables at CT_BITS fractional bits; false if
// an enclosure fails (it does not for the supported ranges).
TMD_HD bool ct_entry(int base, int level, int b, const CoeffConsts& C, uint64_t* lo, uint64_t* hi) {
    using namespace fx;
    Enc<CT_LIMBS> f;
    if (base == 2) {  // log(256 + b) at level 0, log(1 + b 2^-16) at level 1
        if (level == 1 && b > 0) {  // 2 atanh(b / (2^17 + b))
            U<CT_LIMBS> S;
            uint64_t E;
            if (!atanh_ratio<CT_LIMBS>((uint64_t)b, (1ull << 17) + (uint64_t)b, CT_BITS, C.div, S, E)) return false;
            f.lo = S;
            f.hi = S;
            add_u64(f.hi, E);
            mul_u64(f.lo, 2);
            mul_u64(f.hi, 2);
        } else if (level != 0) {  // log 1 and the unused levels
            set_zero(f.lo);
            set_zero(f.hi);
        } else {
            Enc<CT_LIMBS> ln2;
            cf_detail::ln2_at<CT_LIMBS>(C, CT_BITS, ln2.lo, ln2.hi);
            if (!log_enc<CT_LIMBS>(256u + (uint64_t)b, 9, 9, CT_BITS, ln2, C.div, f)) return false;
        }
    } else if (b == 0 || (base == 1 && level == 0)) {  // 1 (level 0 of base 2 is unused)
        set_pow2(f.lo, CT_BITS);
        f.hi = f.lo;
    } else if (base == 0) {
        if (level == 0 && b >= 4) {
            set_zero(f.lo);
            set_zero(f.hi);
        } else if (!exp_small<CT_LIMBS>((uint64_t)b, 8u * (unsigned)level, CT_BITS, C.div, f)) {
            return false;
        }
    } else {
        CoeffJob J;
        J.func = 1;
        J.e_in = 0;
        J.p = 8 * level;  // X = b 2^-(8 level): q = p - e_in = 8 level
        J.d = 0;
        J.L = 1;
        J.scale_log2 = 0;
        J.log2_N = 0;
        J.red = 0;
        if (!exp2_arg<CT_LIMBS>(J, (uint64_t)b, CT_BITS, C, f)) return false;
    }
    for (int i = 0; i < CT_LIMBS; i++) {
        lo[i] = f.lo.w[i];
        hi[i] = f.hi.w[i];
    }
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

// An entry of the tables as NL limbs at PA = 64 (NL - 2) + 60 fractional
// bits (the top NL of its CT_LIMBS limbs; the upper end rounded up).
template <int NL>
TMD_HD void ct_load(const uint64_t* tab, int base, int level, int b, fx::U<NL>& lo, fx::U<NL>& hi) {
    static_assert(NL <= CT_LIMBS, "table entries hold CT_LIMBS limbs");
    const uint64_t* e = tab + ct_index(base, level, b, 0);
#pragma unroll
    for (int i = 0; i < NL; i++) {
        lo.w[i] = e[CT_LIMBS - NL + i];
        hi.w[i] = e[CT_LIMBS + CT_LIMBS - NL + i];
    }
    if (NL < CT_LIMBS) fx::add_u64(hi, 1);
}

// The lower end only (truncated to PA fractional bits).
template <int NL>
TMD_HD void ct_load_lo(const uint64_t* tab, int base, int level, int b, fx::U<NL>& lo) {
    static_assert(NL <= CT_LIMBS, "table entries hold CT_LIMBS limbs");
    const uint64_t* e = tab + ct_index(base, level, b, 0);
#pragma unroll
    for (int i = 0; i < NL; i++) lo.w[i] = e[CT_LIMBS - NL + i];
}

// Enclosure of f(X) 2^-red (exp with red = 0, 2^x) with PB fractional bits
// from the tables: X = n + sum_i b_i 2^(-8 i) (the fraction of X = M 2^-q
// left-aligned to 80 bits), f = e^n prod_i T(0, i, b_i) for exp and
// 2^n prod_i T(1, i, b_i) for 2^x, the products formed at PA fractional bits
// (below CT_LIMBS limbs the lower ends' product and a bound on its error,
// at CT_LIMBS limbs both ends) and shifted to PB bits.  False when the
// tables do not apply (log, exp above [2, 4), more than 80 fractional
// bits), so that the caller takes the series.
// log X for X = M 2^(e_in - p): with g = the top 9 bits of M (256 <= g <
// 512), G = g 2^(p - 9), the next 8 bits h = floor((M - G) / (g 2^(p - 25)))
// (h < 256; h = 0 for p < 25) and M' = G (1 + h 2^-16) = G + g h 2^(p - 25)
// <= M, X = g (1 + h 2^-16) (M / M') 2^(e_in - 9), so
//   log X = log g + log(1 + h 2^-16) + (e_in - 9) ln 2
//           + 2 atanh((M - M') / (M + M')),
// the ratio below 2^-17 (M - M' < G 2^-16): a series of ~P/34 terms instead
// of ~P/3.2 for the direct atanh of (2^p - M)/(2^p + M) <= 1/3.  log g and
// log(1 + h 2^-16) from the tables, ln 2 from the constants, all with PB
// fractional bits (PB + 8 <= PA).
template <int NL>
TMD_HD bool f_table_log(const CoeffJob& J, uint64_t M, unsigned PB, const uint64_t* tab, const CoeffConsts& C,
                        fx::Enc<NL>& f) {
    using namespace fx;
    constexpr unsigned PA = 64u * NL - 68u;
    if (J.p < 9 || J.p > 61) return false;
    const unsigned sh = (unsigned)(J.p - 9);
    const uint64_t g = M >> sh, G = g << sh;
    if (g < 256 || g >= 512) return false;
    uint32_t h = 0;
    uint64_t Mp = G;
    if (J.p >= 25) {
        const unsigned s2 = (unsigned)(J.p - 25);
        h = (uint32_t)((M - G) >> s2) / (uint32_t)g;  // (M - G) >> s2 < 2^16
        Mp = G + (((uint64_t)g * h) << s2);
    }
    U<NL> S;
    uint64_t E;
    if (!atanh_ratio<NL>(M - Mp, M + Mp, PB, C.div, S, E)) return false;
    U<NL> tlo, thi;
    ct_load<NL>(tab, 2, 0, (int)(g - 256), tlo, thi);
    if (h) {
        U<NL> ulo, uhi;
        ct_load<NL>(tab, 2, 1, (int)h, ulo, uhi);
        add(tlo, ulo);
        add(thi, uhi);
    }
    const unsigned s = PA - PB;
    const bool up = low_bits(thi, s);
    shr(tlo, s);
    shr(thi, s);
    if (up) add_u64(thi, 1);
    U<NL> llo, lhi;
    ln2_at<NL>(C, PB, llo, lhi);
    const int e = J.e_in - 9;
    const uint64_t ae = (uint64_t)(e < 0 ? -e : e);
    // lower end: log g (lo) + 2 S +/- |e| ln 2 (lo when adding, hi when subtracting)
    U<NL> lo = tlo, hi = thi, a = S, b = S;
    mul_u64(a, 2);
    add_u64(b, E);
    mul_u64(b, 2);
    add(lo, a);
    add(hi, b);
    U<NL> el = e < 0 ? lhi : llo, eh = e < 0 ? llo : lhi;
    mul_u64(el, ae);
    mul_u64(eh, ae);
    if (e < 0) {
        if (sub(lo, el)) return false;
        if (sub(hi, eh)) return false;
    } else {
        add(lo, el);
        add(hi, eh);
    }
    f.lo = lo;
    f.hi = hi;
    return true;
}

template <int NL>
TMD_HD bool f_table(const CoeffJob& J, uint64_t M, unsigned PB, const uint64_t* tab, const CoeffConsts& C,
                    fx::Enc<NL>& f, bool& exact) {
    using namespace fx;
    constexpr unsigned PA = 64u * NL - 68u;
    exact = false;
    const unsigned q = (unsigned)(J.p - J.e_in);
    if (!tab || PB + 8 > PA) return false;
    if (J.func == 2) return f_table_log<NL>(J, M, PB, tab, C, f);
    if (q > 80) return false;
    if (J.func == 0 && J.red) return false;
    if (J.func == 1) {
        if (J.red) {  // 2^(X - red), X - red = (M - red 2^q) 2^-q in [0, 1)
            if (q == 0 || q >= 64 || (M >> q) != (uint64_t)J.red) return false;
            M -= (uint64_t)J.red << q;
        }
        if (integer_arg(M, q)) {  // 2^X at an integer X
            set_pow2(f.lo, PB + (unsigned)(q >= 64 ? 0 : (M >> q)));
            f.hi = f.lo;
            exact = true;
            return true;
        }
    }
    const uint64_t n = q >= 64 ? 0 : (M >> q);
    if (n > 3) return false;
    const uint64_t F = q >= 64 ? M : (M & ((1ull << q) - 1));
    // the 80-bit left-aligned fraction V = F 2^(80 - q) as (vh, vl)
    uint64_t vh, vl;
    const unsigned sh = 80u - q;
    if (sh >= 64) {
        vh = F << (sh - 64);
        vl = 0;
    } else {
        vl = F << sh;
        vh = sh ? (F >> (64 - sh)) : 0;
    }
    const int base = J.func == 0 ? 0 : 1;
    U<NL> lo, hi;
    if (NL < CT_LIMBS) {
        // One chain, of the lower ends, and a bound for the upper end.  With
        // u = 2^-PA, every lower end t' of a factor t >= 1 (an entry truncated
        // from CT_BITS to PA bits; the entries' own widths are far below u)
        // has t - 2u < t' <= t, and every truncated product x' = mul_trunc(x,
        // t') has x t' - 2u < x' <= x t'.  With P_k the exact product of the
        // first k factors (P_k >= 1) and x_k its lower end,
        //   P_k - x_k <= P_(k-1) (t - t') + (P_(k-1) - x_(k-1)) t + 2u,
        // so (P_k - x_k) / P_k grows by at most 4u per product: at most 42u
        // after the start and ten products, and P < 2^6 (X < 4) gives
        // P - x < 2688u < 2^12 u.
        if (base == 0) {
            ct_load_lo<NL>(tab, 0, 0, (int)n, lo);
        } else {
            set_pow2(lo, PA + (unsigned)n);
        }
#pragma unroll 1
        for (int i = 1; i <= 10; i++) {
            const unsigned pos = 80u - 8u * (unsigned)i;  // bits [pos, pos + 8) of V
            const unsigned b = pos >= 64 ? (unsigned)(vh >> (pos - 64)) & 255u
                                         : (unsigned)((vl >> pos) | (pos > 56 ? vh << (64 - pos) : 0)) & 255u;
            if (b == 0) continue;
            U<NL> t, r;
            ct_load_lo<NL>(tab, base, i, (int)b, t);
            mul_trunc<NL>(lo, t, r);
            lo = r;
        }
        hi = lo;
        add_u64(hi, 1ull << 12);
    } else {
        // at the entries' own width: both ends, each product's upper end
        // raised by two units
        if (base == 0) {
            ct_load<NL>(tab, 0, 0, (int)n, lo, hi);
        } else {
            set_pow2(lo, PA + (unsigned)n);
            hi = lo;
        }
#pragma unroll 1
        for (int i = 1; i <= 10; i++) {
            const unsigned pos = 80u - 8u * (unsigned)i;
            const unsigned b = pos >= 64 ? (unsigned)(vh >> (pos - 64)) & 255u
                                         : (unsigned)((vl >> pos) | (pos > 56 ? vh << (64 - pos) : 0)) & 255u;
            if (b == 0) continue;
            U<NL> tlo, thi, r;
            ct_load<NL>(tab, base, i, (int)b, tlo, thi);
            mul_trunc<NL>(lo, tlo, r);
            lo = r;
            mul_trunc<NL>(hi, thi, r);
            hi = r;
            add_u64(hi, 2);
        }
    }
    const unsigned s = PA - PB;
    const bool up = low_bits(hi, s);
    shr(lo, s);
    shr(hi, s);
    if (up) add_u64(hi, 1);
    f.lo = lo;
    f.hi = hi;
    return true;
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

// c[k*COEFF_MAX_LIMBS + l] for k = 0..d, l < L (limb l of c_k; the other
// slots zero).  Returns false when a rounding stays undecided at this width
// (retry with a wider NL) or a width is exceeded.  With the device tables
// f(X_t) comes from their products, with an anchor of the block's job from
// the anchored short series, else from the direct series.  (The order and
// table-word loops stay rolled: unrolled to the largest degree they keep the
// coefficients in registers but make the table kernel, one or two warps per
// SM on small plans, wait on instruction fetches -- 44 against 63 us on the
// 4096 blocks of a 2^36-argument slice.)  With step > 1 the caller splits
// the orders over `step` threads: this one writes the slots of the orders k
// = part (mod step), every thread running the same code on its own order (f
// and the chains of 2^x and log, up to its order, are formed by each).
template <int NL>
TMD_HD bool block_coeffs(const CoeffJob& J, uint64_t M, int guard, const CoeffConsts& C, uint64_t* c,
                         const Anchor* anchor = nullptr, const uint64_t* tables = nullptr, int part = 0,
                         int step = 1) {
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
    if (!(tables && cf_detail::f_table<NL>(J, M, PB, tables, C, f, exact)))
        if (!(anchor && !integer_x && cf_detail::f_anchored<NL>(J, M, PB, C, *anchor, f)))
            if (!cf_detail::f_direct<NL>(J, M, PB, C, f, exact)) return false;
    if (J.func == 2) {  // log
        const int s = (int)P - E0;
        if (s < 1) return false;
        cf_detail::rn_shift(f.lo, (unsigned)s);
        cf_detail::rn_shift(f.hi, (unsigned)s);
        if (!equal(f.lo, f.hi)) return false;
        if (part == 0) cf_detail::store_mod_w(f.lo, false, J.L, c);
        // the order-k coefficient's scale 2^(E0 + k (e_in - p)) times the
        // k-th power of the argument's 2^(p - e_in) leaves 2^E0 for every k
        return cf_detail::log_orders<NL>(M, J.d, E0, C, J.L, c, part, step);
    }
    // exp or 2^x: the enclosure of f(X_t) has P2 = PB fractional bits
    const unsigned P2 = PB;
    U<NL> l2lo, l2hi;
    if (J.func == 1) cf_detail::ln2_at<NL>(C, P2, l2lo, l2hi);
    U<NL> plo = f.lo, phi = f.hi;  // f (ln 2)^k enclosure, updated per order
    // 2^x: one chain of lower ends x_k = floor(x_(k-1) l / 2^P2), l the lower
    // ln 2 (l <= L2 = 2^P2 ln 2 < l + 2), and a bound w_k on the distance of
    // x_k to v_k = 2^P2 f (ln 2)^k instead of a second chain: v_k - x_k <=
    // (v_(k-1) (L2 - l) + (v_(k-1) - x_(k-1)) l) / 2^P2 + 1 < 2 Bf + (3/4)
    // w_(k-1) + 1 with f < Bf, starting from the width of f's enclosure
    // (both ends kept when that width or f is too large for the bound)
    bool one_chain = false;
    uint64_t wk = 0, Bf2 = 0;
    if (J.func == 1) {
        U<NL> wd = f.hi;
        sub(wd, f.lo);
        const unsigned fb = bit_length(f.hi);
        if (bit_length(wd) <= 32 && fb <= P2 + 32) {
            one_chain = true;
            wk = wd.w[0];
            Bf2 = 2ull << (fb > P2 ? fb - P2 : 0);
        }
    }
    int have = 0;  // factors of ln 2 applied to (plo, phi)
#pragma unroll 1
    for (int k = part; k <= COEFF_MAX_DEG; k += step) {
        if (k > J.d) {
#pragma unroll
            for (int l = 0; l < COEFF_MAX_LIMBS; l++) c[k * COEFF_MAX_LIMBS + l] = 0;
            continue;
        }
#pragma unroll 1
        while (J.func == 1 && have < k) {
            have++;
            U<NL> t;
            mul_shr(plo, l2lo, P2, t);
            plo = t;
            if (one_chain) {
                wk = wk - wk / 4 + Bf2 + 2;
                phi = plo;
                add_u64(phi, wk);
            } else {
                // upper end: ceil of the product
                U<NL> hprod;
                mul_shr(phi, l2hi, P2, hprod);
                add_u64(hprod, 1);
                phi = hprod;
            }
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
#pragma unroll
            for (int l = 0; l < COEFF_MAX_LIMBS; l++) c[k * COEFF_MAX_LIMBS + l] = 0;
            continue;
        }
        cf_detail::rn_shift(lo, (unsigned)s);
        cf_detail::rn_shift(hi, (unsigned)s);
        if (!equal(lo, hi)) return false;
        cf_detail::store_mod_w(lo, false, J.L, c + k * COEFF_MAX_LIMBS);
    }
    (void)exact;
    return true;
}

// The 2d+1 table words from the coefficients c[k*COEFF_MAX_LIMBS + l]: w =
// 0..d are Delta^w g0(0) with g0(i) = R(iN), w = d+1..2d are
// Delta^(w-d-1) g1(0) with g1(i) = R(iN+1) - R(iN), all mod 2^W; table[w*L +
// l].  Closed forms instead of values and differences: as polynomials in i,
// g0(i) = sum_j a_j i^j with a_j = c_j N^j, and g1(i) = sum_{j<d} b_j i^j
// with b_j = N^j sum_{k>j} C(k, j) c_k (R shifted by one, less R).  The
// w-th forward difference of i^j at i = 0 is w! S(j, w) (S the Stirling
// numbers of the second kind; w! S(j, w) counts the maps of a j-set onto a
// w-set), so
//     Delta^w g0(0) = sum_{j>=w} a_j w! S(j, w),
//     Delta^w g1(0) = sum_{j>=w} b_j w! S(j, w).
// Every step is a ring operation, so the words equal the differences of the
// values mod 2^W exactly; N^j is a shift.  The coefficients above d are zero.
// With step > 1 this thread writes the words w = part (mod step), each by the
// same code with its own constants (block_table_words_split).
namespace cf_detail {
// acc += m x (mod 2^(64 COEFF_MAX_LIMBS)) for a small constant m
TMD_HD void add_mul_small(fx::U<COEFF_MAX_LIMBS>& acc, const fx::U<COEFF_MAX_LIMBS>& x, uint32_t m) {
    if (m == 0) return;
    if (m == 1) {
        fx::add(acc, x);
        return;
    }
    fx::U<COEFF_MAX_LIMBS> t = x;
    fx::mul_u64(t, m);
    fx::add(acc, t);
}
}  // namespace cf_detail

TMD_HD void block_table_words_split(const CoeffJob& J, const uint64_t* c, uint64_t* table, int part, int step);

TMD_HD void block_table_words(const CoeffJob& J, const uint64_t* c, uint64_t* table, int part = 0, int step = 1) {
    if (step > 1) {
        block_table_words_split(J, c, table, part, step);
        return;
    }
    using namespace fx;
    using V = U<COEFF_MAX_LIMBS>;
    constexpr int D = COEFF_MAX_DEG;
    static_assert(D == 4, "the constants below cover degrees up to 4");
    // binom[k][j] = C(k, j); surj[j][w] = w! S(j, w)
    constexpr uint32_t binom[D + 1][D + 1] = {
        {1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0}, {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};
    constexpr uint32_t surj[D + 1][D + 1] = {
        {1, 0, 0, 0, 0}, {0, 1, 0, 0, 0}, {0, 1, 2, 0, 0}, {0, 1, 6, 6, 0}, {0, 1, 14, 36, 24}};
    const int L = J.L, d = J.d;
    const unsigned lg = (unsigned)J.log2_N;
    V ck[D + 1], a[D + 1], b[D];
#pragma unroll
    for (int k = 0; k <= D; k++)
#pragma unroll
        for (int l = 0; l < COEFF_MAX_LIMBS; l++) ck[k].w[l] = c[k * COEFF_MAX_LIMBS + l];
#pragma unroll
    for (int j = 0; j <= D; j++) {
        a[j] = ck[j];
        shl(a[j], (unsigned)j * lg);
    }
#pragma unroll
    for (int j = 0; j < D; j++) {
        set_zero(b[j]);
#pragma unroll
        for (int k = j + 1; k <= D; k++) cf_detail::add_mul_small(b[j], ck[k], binom[k][j]);
        shl(b[j], (unsigned)j * lg);
    }
#pragma unroll
    for (int w = 0; w <= D; w++) {
        if (w > d) break;
        V t;
        set_zero(t);
#pragma unroll
        for (int j = w; j <= D; j++) cf_detail::add_mul_small(t, a[j], surj[j][w]);
#pragma unroll
        for (int l = 0; l < COEFF_MAX_LIMBS; l++)
            if (l < L) table[w * L + l] = t.w[l];
    }
#pragma unroll
    for (int w = 0; w < D; w++) {
        if (w >= d) break;
        V t;
        set_zero(t);
#pragma unroll
        for (int j = w; j < D; j++) cf_detail::add_mul_small(t, b[j], surj[j][w]);
#pragma unroll
        for (int l = 0; l < COEFF_MAX_LIMBS; l++)
            if (l < L) table[(d + 1 + w) * L + l] = t.w[l];
    }
}

// The words w = part (mod step) of block_table_words, every word by the same
// code: the sums run over all j with the multipliers w! S(j, w) (zero for j <
// w) read from packed constants, g0's or g1's coefficients selected per word.
TMD_HD void block_table_words_split(const CoeffJob& J, const uint64_t* c, uint64_t* table, int part, int step) {
    using namespace fx;
    using V = U<COEFF_MAX_LIMBS>;
    constexpr int D = COEFF_MAX_DEG;
    static_assert(D == 4, "the constants below cover degrees up to 4");
    // byte w of SURJ[j] is w! S(j, w)
    constexpr uint64_t SURJ[D + 1] = {0x01ull, 0x0100ull, 0x020100ull, 0x06060100ull, 0x18240E0100ull};
    constexpr uint32_t binom[D + 1][D + 1] = {
        {1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0}, {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};
    const int L = J.L, d = J.d;
    const unsigned lg = (unsigned)J.log2_N;
    V ck[D + 1], a[D + 1], b[D + 1];
#pragma unroll
    for (int k = 0; k <= D; k++)
#pragma unroll
        for (int l = 0; l < COEFF_MAX_LIMBS; l++) ck[k].w[l] = c[k * COEFF_MAX_LIMBS + l];
#pragma unroll
    for (int j = 0; j <= D; j++) {
        a[j] = ck[j];
        shl(a[j], (unsigned)j * lg);
        set_zero(b[j]);
#pragma unroll
        for (int k = j + 1; k <= D; k++) cf_detail::add_mul_small(b[j], ck[k], binom[k][j]);
        shl(b[j], (unsigned)j * lg);
    }
#pragma unroll 1
    for (int om = part; om <= 2 * d; om += step) {
        const bool g0 = om <= d;
        const unsigned w = (unsigned)(g0 ? om : om - d - 1);
        V t;
        set_zero(t);
#pragma unroll
        for (int j = 0; j <= D; j++) {
            V x;
#pragma unroll
            for (int l = 0; l < COEFF_MAX_LIMBS; l++) x.w[l] = g0 ? a[j].w[l] : b[j].w[l];
            mul_u64(x, (SURJ[j] >> (8u * w)) & 0xffu);
            add(t, x);
        }
#pragma unroll
        for (int l = 0; l < COEFF_MAX_LIMBS; l++)
            if (l < L) table[om * L + l] = t.w[l];
    }
}

// The coefficients in the order of the external tables: out[k*L + l].
TMD_HD void coeffs_packed(const CoeffJob& J, const uint64_t* c, uint64_t* out) {
#pragma unroll
    for (int k = 0; k <= COEFF_MAX_DEG; k++) {
        if (k > J.d) break;
#pragma unroll
        for (int l = 0; l < COEFF_MAX_LIMBS; l++)
            if (l < J.L) out[k * J.L + l] = c[k * COEFF_MAX_LIMBS + l];
    }
}

}  // namespace tmd
