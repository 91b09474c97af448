// Host-side part of the generation stage: validation, output-binade cuts,
// block plan, correctly rounded Taylor coefficients and difference tables.
//
// Values of f are enclosed in fixed point with P fractional bits,
// lo/2^P <= value <= hi/2^P, from power series summed with truncating
// arithmetic plus an explicit bound on the accumulated truncation and on the
// series tail.  A coefficient is accepted only when both ends of its
// enclosure round to the same integer; otherwise P grows (Ziv's strategy).
#include "host.hpp"

#include <algorithm>
#include <cmath>
#include <cstring>

#include "bigint.hpp"
#include "coeffs.cuh"

namespace tmd {

namespace {

struct Enc {
    Big lo, hi;      // lo / 2^P <= value <= hi / 2^P
    unsigned P;
};

// exp(y / 2^Q), y >= 0, with P fractional bits.
// t_0 = 2^P, t_n = floor(t_{n-1} X / n); the truncation error e_n of t_n
// obeys e_n <= e_{n-1} X / n + 1, tracked with X <= Xc = ceil(X).  Once
// t_n = 0 with n >= 2 Xc + 2, the true term is at most e_n and the tail after
// it at most the term itself (ratio X/(n+1) < 1/2).
Enc exp_fixed(const Big& y, unsigned Q, unsigned P) {
    Big yc = y;
    yc.add(Big::pow2(Q).sub(Big(1)));
    yc.shr(Q);
    uint64_t Xc = yc.limb(0);
    Big t = Big::pow2(P);
    Big S = t;
    uint64_t e = 0, E = 0;
    for (uint64_t n = 1;; n++) {
        t = Big::mul(t, y);
        t.shr(Q);
        t.div_u64(n);
        e = (e * Xc + n - 1) / n + 1;
        S.add(t);
        E += e;
        if (t.zero() && n >= 2 * Xc + 2) {
            E += e + 1;
            break;
        }
    }
    Enc r;
    r.lo = S;
    r.hi = S;
    r.hi.add(Big(E));
    r.P = P;
    return r;
}

// ln 2 = sum_k 2 / ((2k+1) 3^(2k+1)):  w_0 = floor(2^(P+1)/3),
// w_k = floor(w_{k-1}/9) (error <= 2), term_k = floor(w_k/(2k+1)) (error <= 2).
Enc ln2_series(unsigned P) {
    Big w = Big::pow2(P + 1);
    w.div_u64(3);
    Big S = w;
    uint64_t E = 1;
    for (uint64_t k = 1;; k++) {
        w.div_u64(9);
        Big t = w;
        t.div_u64(2 * k + 1);
        S.add(t);
        E += 2;
        if (t.zero()) {
            E += 1;
            break;
        }
    }
    Enc r;
    r.lo = S;
    r.hi = S;
    r.hi.add(Big(E));
    r.P = P;
    return r;
}

// ln 2 enclosures are reused across blocks: one cache per host thread.
Enc ln2_fixed(unsigned P) {
    thread_local std::vector<std::pair<unsigned, Enc>> cache;
    for (const auto& e : cache)
        if (e.first == P) return e.second;
    Enc r = ln2_series(P);
    if (cache.size() > 32) cache.clear();
    cache.emplace_back(P, r);
    return r;
}

// 2^X with X = M / 2^q: exact at integers, else exp(X ln 2) with the argument
// enclosed from both sides (exp is increasing).
Enc exp2_fixed(uint64_t M, unsigned q, unsigned P) {
    Enc r;
    r.P = P;
    if (integer_arg(M, q)) {
        uint64_t X = q >= 64 ? 0 : (M >> q);
        r.lo = Big::pow2(P + (unsigned)X);
        r.hi = r.lo;
        return r;
    }
    unsigned P2 = P + 16;
    Enc L = ln2_fixed(P2);
    Big ylo = L.lo;
    ylo.mul_u64(M);
    ylo.shr(q);
    Big yhi = L.hi;
    yhi.mul_u64(M);
    yhi = shr_ceil(yhi, q);
    r.lo = exp_fixed(ylo, P2, P).lo;
    r.hi = exp_fixed(yhi, P2, P).hi;
    return r;
}

// log X for X = M 2^(e_in - p), 2^(p-1) <= M < 2^p, e_in >= 2:
// log X = e_in ln 2 - 2 atanh(z), z = (2^p - M) / (2^p + M) in (0, 1/3].
// w_0 = floor(2^P num/den) (error <= 1); w_k = w_{k-1} z^2 by two
// truncating multiply-divides (error <= e/9 + 2 <= 3); term_k =
// floor(w_k / (2k+1)) (error <= 2); tail after a zero term <= 1.
Enc log_fixed(uint64_t M, int p, int e_in, unsigned P) {
    uint64_t num = (1ull << p) - M, den = (1ull << p) + M;
    Big w = Big::pow2(P);
    w.mul_u64(num);
    w.div_u64(den);
    Big S = w;
    uint64_t E = 1;
    for (uint64_t k = 1;; k++) {
        w.mul_u64(num);
        w.div_u64(den);
        w.mul_u64(num);
        w.div_u64(den);
        Big t = w;
        t.div_u64(2 * k + 1);
        S.add(t);
        E += 2;
        if (t.zero()) {
            E += 1;
            break;
        }
    }
    Enc L = ln2_fixed(P);
    Enc r;
    r.P = P;
    Big two_hi = S;
    two_hi.add(Big(E));
    two_hi.mul_u64(2);
    Big two_lo = S;
    two_lo.mul_u64(2);
    r.lo = L.lo;
    r.lo.mul_u64((uint64_t)e_in);
    r.lo.sub(two_hi);
    r.hi = L.hi;
    r.hi.mul_u64((uint64_t)e_in);
    r.hi.sub(two_lo);
    return r;
}

uint64_t factorial(int k) {
    uint64_t r = 1;
    for (int i = 2; i <= k; i++) r *= (uint64_t)i;
    return r;
}

// Enclosure of f^(k)(X)/k! (k = 0: f itself) for the positive cases:
// exp (any k), 2^x (any k), log (k = 0).  X = M 2^(e_in - p).  `base`, when
// given, is an enclosure of f(X) (exp, 2^x) at precision base->P >= the
// precision this order needs; it is reused instead of summing the series
// again.
Enc coeff_enclosure(int func, uint64_t M, int p, int e_in, int k, unsigned P,
                    const Enc* base = nullptr) {
    unsigned q = (unsigned)(p - e_in);
    uint64_t kf = factorial(k);
    Enc r;
    if (func == TMD_EXP) {
        if (base && base->P >= P) {
            r.lo = base->lo;
            r.lo.shr(base->P - P);
            r.hi = shr_ceil(base->hi, base->P - P);
            r.P = P;
        } else {
            r = exp_fixed(Big(M), q, P);
        }
    } else if (func == TMD_EXP2) {
        unsigned P2 = P + 8 + 2 * (unsigned)k;
        Enc e;
        if (base && base->P >= P2) {
            e.lo = base->lo;
            e.lo.shr(base->P - P2);
            e.hi = shr_ceil(base->hi, base->P - P2);
            e.P = P2;
        } else {
            e = exp2_fixed(M, q, P2);
        }
        if (k > 0) {
            Enc L = ln2_fixed(P2);
            Big lo = e.lo, hi = e.hi;
            for (int i = 0; i < k; i++) {
                lo = Big::mul(lo, L.lo);
                lo.shr(P2);
                hi = Big::mul(hi, L.hi);
                hi = shr_ceil(hi, P2);
            }
            e.lo = lo;
            e.hi = hi;
        }
        r.lo = e.lo;
        r.lo.shr(P2 - P);
        r.hi = shr_ceil(e.hi, P2 - P);
        r.P = P;
    } else {
        r = log_fixed(M, p, e_in, P);
    }
    if (kf > 1) {
        r.lo.div_u64(kf);
        uint64_t rem = r.hi.div_u64(kf);
        if (rem) r.hi.add_u64(1);
    }
    return r;
}

// RN(v) = floor(v + 1/2) of v = x / 2^s for x >= 0 (s >= 1).
Big rn_shift(const Big& x, unsigned s) {
    Big t = x;
    t.add(Big::pow2(s - 1));
    t.shr(s);
    return t;
}

// Signed result of RN(2^E f^(k)(X)/k!) reduced mod 2^W into `limbs` words.
// `base` (optional) is a shared enclosure of f(X) for exp and 2^x.
bool scaled_coeff(int func, uint64_t M, int p, int e_in, int k, int E, unsigned limbs,
                  uint64_t* out, const Enc* base = nullptr) {
    Big mag;
    bool neg = false;
    if (func == TMD_LOG && k >= 1) {
        // exact rational: (-1)^(k-1) 2^(E + k q) / (k M^k)
        int q = p - e_in;
        int sh = E + k * q;
        if (sh < 0) return false;
        neg = (k % 2) == 0;
        Big den = Big((uint64_t)k);
        for (int i = 0; i < k; i++) den.mul_u64(M);
        Big x = Big::pow2((unsigned)sh + 1);
        x.add(den);
        if (neg) x.sub(Big(1));
        // floor((2 num + den [- 1]) / (2 den)) by a chain of exact floors
        x.div_u64(2);
        x.div_u64((uint64_t)k);
        for (int i = 0; i < k; i++) x.div_u64(M);
        mag = x;
    } else {
        bool done = false;
        for (int step = 0; step < 16 && !done; step++) {
            int e_pos = E > 0 ? E : 0;
            unsigned P = (unsigned)(e_pos + 64 + 64 * step);
            Enc c = coeff_enclosure(func, M, p, e_in, k, P, step == 0 ? base : nullptr);
            int s = (int)P - E;
            if (s < 1) continue;
            Big rl = rn_shift(c.lo, (unsigned)s);
            Big rh = rn_shift(c.hi, (unsigned)s);
            if (rl.cmp(rh) == 0) {
                mag = rl;
                done = true;
            }
        }
        if (!done) return false;
    }
    // reduce mod 2^W, negate in two's complement if needed
    uint64_t w[MAX_LIMBS] = {0, 0, 0};
    for (unsigned l = 0; l < limbs; l++) w[l] = mag.limb(l);
    if (neg) {
        uint64_t c = 1;
        for (unsigned l = 0; l < limbs; l++) {
            uint64_t x = ~w[l];
            w[l] = x + c;
            c = (w[l] < x) ? 1 : 0;
        }
    }
    for (unsigned l = 0; l < limbs; l++) out[l] = w[l];
    return true;
}

// ---- W-bit words (mod 2^W), little-endian limbs ----
struct Word {
    uint64_t l[MAX_LIMBS];
};

Word w_zero() {
    Word r;
    memset(&r, 0, sizeof r);
    return r;
}
Word w_add(const Word& a, const Word& b, unsigned L) {
    Word r = w_zero();
    uint64_t c = 0;
    for (unsigned i = 0; i < L; i++) {
        u128 s = (u128)a.l[i] + b.l[i] + c;
        r.l[i] = (uint64_t)s;
        c = (uint64_t)(s >> 64);
    }
    return r;
}
Word w_sub(const Word& a, const Word& b, unsigned L) {
    Word r = w_zero();
    uint64_t br = 0;
    for (unsigned i = 0; i < L; i++) {
        u128 d = (u128)a.l[i] - b.l[i] - br;
        r.l[i] = (uint64_t)d;
        br = (uint64_t)(d >> 64) ? 1 : 0;
    }
    return r;
}
Word w_mul_u64(const Word& a, uint64_t m, unsigned L) {
    Word r = w_zero();
    uint64_t c = 0;
    for (unsigned i = 0; i < L; i++) {
        u128 p = (u128)a.l[i] * m + c;
        r.l[i] = (uint64_t)p;
        c = (uint64_t)(p >> 64);
    }
    return r;
}
// R(y) = sum_k c_k y^k mod 2^W by Horner's rule
Word horner(const Word* c, int d, uint64_t y, unsigned L) {
    Word acc = c[d];
    for (int k = d - 1; k >= 0; k--) acc = w_add(w_mul_u64(acc, y, L), c[k], L);
    return acc;
}

// f(X) enclosure used for the output exponent
Enc f_enclosure(const tmd_job& job, uint64_t M, unsigned P) {
    return coeff_enclosure(job.func, M, job.p, job.e_in, 0, P);
}

uint64_t arg_mantissa(const tmd_job& job, uint64_t j) { return (1ull << (job.p - 1)) + j; }

// First j (possibly outside the slice) with e(f(X_j)) >= e, by the inverse
// function: f(X) >= 2^(e-1) iff X >= t_e with t_e = (e-1) ln 2 (exp),
// e - 1 (2^x), exp(2^(e-1)) (log).  X_j = M_j 2^-q, so the cut is
// ceil(t_e 2^q) - 2^(p-1); t_e 2^q is irrational except for 2^x.
bool cut_index(const tmd_job& job, int e, int64_t* out) {
    int q = job.p - job.e_in;
    int64_t half = (int64_t)1 << (job.p - 1);
    if (job.func == TMD_EXP2) {
        if (q >= 62) return false;  // a cut needs X >= 1: q <= p - 1 there
        *out = (int64_t)(e - 1) * ((int64_t)1 << q) - half;
        return true;
    }
    for (unsigned P = (unsigned)q + 96; P < (unsigned)q + 96 + 64 * 12; P += 64) {
        Big lo, hi;
        if (job.func == TMD_EXP) {
            if (e - 1 <= 0) return false;
            Enc L = ln2_fixed(P);
            lo = L.lo;
            lo.mul_u64((uint64_t)(e - 1));
            hi = L.hi;
            hi.mul_u64((uint64_t)(e - 1));
        } else {
            Enc x;
            if (e - 1 >= 0)
                x = exp_fixed(Big(1ull << (e - 1)), 0, P);
            else
                x = exp_fixed(Big(1), (unsigned)(1 - e), P);
            lo = x.lo;
            hi = x.hi;
        }
        // floor(value 2^q) = floor(lo / 2^(P - q))
        lo.shr(P - (unsigned)q);
        hi.shr(P - (unsigned)q);
        if (lo.cmp(hi) == 0) {
            if (lo.v.size() > 1) return false;
            *out = (int64_t)lo.limb(0) + 1 - half;
            return true;
        }
    }
    return false;
}

}  // namespace

tmd_status validate_job(const tmd_job& job) {
    if (job.reserved != 0) return TMD_EINVAL;
    if (job.func < TMD_EXP || job.func > TMD_LOG) return TMD_EINVAL;
    if (job.p < 8 || job.p > 60) return TMD_EUNSUPPORTED;
    if (job.m < 2 || job.m > 63) return TMD_EINVAL;
    if (job.log2_N < 1 || job.log2_N > 16) return TMD_EUNSUPPORTED;
    if (job.log2_T < job.log2_N || job.log2_T > 40) return TMD_EINVAL;
    if (job.log2_T - job.log2_N > 16) return TMD_EUNSUPPORTED;
    if (job.d < 1 || job.d > MAX_DEG) return TMD_EUNSUPPORTED;
    if (job.limbs < 1 || job.limbs > MAX_LIMBS) return TMD_EUNSUPPORTED;
    if (job.flags & ~(uint32_t)(TMD_BP_DIRECTED | TMD_ALL_HITS | TMD_LEFEVRE | TMD_SOUND)) return TMD_EINVAL;
    if (job.flags & TMD_SOUND) {
        if (job.flags & TMD_ALL_HITS) return TMD_EINVAL;
        if (job.eps3 < (1ull << (64 - job.m)) || job.eps1 >= (1ull << 62) ||
            job.eps1 < job.eps3 + (1ull << job.log2_N) + 2)
            return TMD_EINVAL;
    } else if (job.eps1 || job.eps3) {
        return TMD_EINVAL;
    }
    if (job.func == TMD_LOG) {
        if (job.e_in < 2 || job.e_in > 16) return TMD_EUNSUPPORTED;
    } else {
        // up to [256, 512): the last binade of exp below binary64's overflow
        if (job.e_in < -16 || job.e_in > 9) return TMD_EUNSUPPORTED;
    }
    // arguments X = M 2^-(p - e_in) with a positive shift; the range-reduced
    // binades (exp, 2^x above [2, 4)) keep at least 8 fractional bits
    if (job.p - job.e_in < 1) return TMD_EUNSUPPORTED;
    if (job.func != TMD_LOG && job.e_in > 2 && job.p - job.e_in < 8) return TMD_EUNSUPPORTED;
    uint64_t span = 1ull << (job.p - 1);
    if (job.count == 0 || job.start >= span || job.count > span - job.start) return TMD_EINVAL;
    // the sub-interval numbering of a job must fit 32 bits
    if ((job.count >> job.log2_N) + (job.count >> job.log2_T) + 8 >= (1ull << 32)) return TMD_EUNSUPPORTED;
    return TMD_OK;
}

// e(exp(X)) = K + 1 for the K with K ln 2 <= X < (K + 1) ln 2, X = M 2^-q:
// K from a double estimate, confirmed on the exact fixed-point X against a
// 192-bit enclosure of ln 2 (false when X is too close to a multiple of ln 2
// to decide there).
bool exp_exponent_reduced(uint64_t M, unsigned q, int* e) {
    const CoeffConsts& C = coeff_consts();
    const unsigned P = 192;
    fx::U<5> llo, lhi, x;
    cf_detail::ln2_at<5>(C, P, llo, lhi);
    fx::set_zero(x);
    x.w[0] = M;
    fx::shl(x, P - q);
    const double est = std::floor(std::ldexp((double)M, -(int)q) / 0.69314718055994530942);
    for (int dk = -1; dk <= 1; dk++) {
        const double kd = est + dk;
        if (kd < 0 || kd > 4096) continue;
        const uint64_t K = (uint64_t)kd;
        fx::U<5> a = lhi, b = llo;
        fx::mul_u64(a, K);       // >= K ln 2
        fx::mul_u64(b, K + 1);   // <= (K + 1) ln 2
        fx::U<5> t = x;
        const bool ge = fx::sub(t, a) == 0;          // X >= K ln2_hi
        fx::U<5> u = b;
        const bool lt = fx::sub(u, x) == 0 && !fx::is_zero(u);  // X < (K+1) ln2_lo
        if (ge && lt) {
            *e = (int)K + 1;
            return true;
        }
    }
    return false;
}

// e(f(X)) from a 128-bit enclosure of f(X) (fixed-size routines, no heap);
// the rare undecided case (f(X) within 2^-100 of a power of two) falls back
// to wider Big enclosures.
bool output_exponent_fx(const tmd_job& job, uint64_t M, int* e) {
    const CoeffConsts& C = coeff_consts();
    const unsigned P = 128, q = (unsigned)(job.p - job.e_in);
    if (job.func == TMD_EXP2 && job.e_in > 2) {  // 2^X in [2^n, 2^(n+1)), n = floor(X)
        *e = (int)(M >> q) + 1;
        return true;
    }
    if (job.func == TMD_EXP && job.e_in > 2) return exp_exponent_reduced(M, q, e);
    fx::Enc<6> f;
    if (job.func == TMD_EXP) {
        if (!fx::exp_small<6>(M, q, P, C.div, f)) return false;
    } else if (job.func == TMD_EXP2) {
        if (integer_arg(M, q)) {
            fx::set_pow2(f.lo, P + (unsigned)(q >= 64 ? 0 : (M >> q)));
            f.hi = f.lo;
        } else {
            fx::U<6> llo, lhi;
            fx::U<LN2_LIMBS> a = C.ln2_lo, b = C.ln2_hi;
            fx::shr(a, LN2_BITS - (P + 16));
            fx::shr(b, LN2_BITS - (P + 16));
            fx::add_u64(b, 1);
            for (int i = 0; i < 6; i++) {
                llo.w[i] = a.w[i];
                lhi.w[i] = b.w[i];
            }
            fx::mul_u64(llo, M);
            fx::shr(llo, q);
            fx::mul_u64(lhi, M);
            fx::shr(lhi, q);
            fx::add_u64(lhi, 1);
            const uint64_t Xc = (uint64_t)1 << (job.e_in > 0 ? job.e_in : 0);
            uint64_t elo, ehi;
            fx::U<6> vlo, vhi;
            if (!fx::exp_big<6>(llo, P + 16, Xc, C.div, vlo, elo)) return false;
            if (!fx::exp_big<6>(lhi, P + 16, Xc, C.div, vhi, ehi)) return false;
            fx::add_u64(vhi, ehi);
            fx::shr(vlo, 16);
            fx::shr(vhi, 16);
            fx::add_u64(vhi, 1);
            f.lo = vlo;
            f.hi = vhi;
        }
    } else {
        fx::Enc<6> ln2;
        fx::U<LN2_LIMBS> a = C.ln2_lo, b = C.ln2_hi;
        fx::shr(a, LN2_BITS - P);
        fx::shr(b, LN2_BITS - P);
        fx::add_u64(b, 1);
        for (int i = 0; i < 6; i++) {
            ln2.lo.w[i] = a.w[i];
            ln2.hi.w[i] = b.w[i];
        }
        if (!fx::log_enc<6>(M, job.p, job.e_in, P, ln2, C.div, f)) return false;
    }
    const int elo = (int)fx::bit_length(f.lo) - (int)P;
    const int ehi = (int)fx::bit_length(f.hi) - (int)P;
    if (elo != ehi) return false;
    *e = elo;
    return true;
}

int output_exponent(const tmd_job& job, uint64_t j) {
    uint64_t M = arg_mantissa(job, j);
    int e;
    if (output_exponent_fx(job, M, &e)) return e;
    for (unsigned P = 64; P < 64 * 20; P += 64) {
        Enc f = f_enclosure(job, M, P);
        int elo = (int)f.lo.bits() - (int)P;
        int ehi = (int)f.hi.bits() - (int)P;
        if (elo == ehi) return elo;
    }
    return 0x7fffffff;
}

tmd_status plan_segments(const tmd_job& job, std::vector<Segment>& segs) {
    segs.clear();
    uint64_t a = job.start, b = job.start + job.count;
    int e0 = output_exponent(job, a);
    int e1 = output_exponent(job, b - 1);
    if (e0 == 0x7fffffff || e1 == 0x7fffffff) return TMD_EUNSUPPORTED;
    if (e1 - e0 + 1 > MAX_SEGMENTS) return TMD_EUNSUPPORTED;
    uint64_t cur = a;
    int e = e0;
    for (int en = e0 + 1; en <= e1; en++) {
        int64_t c;
        if (!cut_index(job, en, &c)) return TMD_EUNSUPPORTED;
        if (c <= (int64_t)cur || c >= (int64_t)b) return TMD_EUNSUPPORTED;
        // the cut must be the first argument with the new exponent
        if (output_exponent(job, (uint64_t)c) != en || output_exponent(job, (uint64_t)c - 1) != en - 1)
            return TMD_EUNSUPPORTED;
        segs.push_back(Segment{cur, (uint64_t)c, e});
        cur = (uint64_t)c;
        e = en;
    }
    segs.push_back(Segment{cur, b, e});
    return TMD_OK;
}

void plan_counts(const tmd_job& job, const std::vector<Segment>& segs, uint64_t* n_blocks,
                 uint64_t* n_subints) {
    uint64_t T = 1ull << job.log2_T, N = 1ull << job.log2_N;
    uint64_t nb = 0, ns = 0;
    for (const Segment& s : segs) {
        uint64_t len = s.j1 - s.j0;
        uint64_t full = len / T, rest = len % T;
        nb += full + (rest ? 1 : 0);
        ns += full * (T / N) + (rest + N - 1) / N;
    }
    *n_blocks = nb;
    *n_subints = ns;
}

bool plan_block(const tmd_job& job, const std::vector<Segment>& segs, uint64_t b, BlockPlan* out) {
    uint64_t T = 1ull << job.log2_T, N = 1ull << job.log2_N;
    uint64_t sub = 0;
    for (const Segment& s : segs) {
        uint64_t len = s.j1 - s.j0;
        uint64_t nb = (len + T - 1) / T;
        if (b < nb) {
            out->start = s.j0 + b * T;
            out->length = (b + 1 < nb) ? T : len - b * T;
            out->first_sub = sub + b * (T / N);
            out->e_out = s.e_out;
            return true;
        }
        b -= nb;
        uint64_t full = len / T, rest = len % T;
        sub += full * (T / N) + (rest + N - 1) / N;
    }
    return false;
}

int scale_log2(const tmd_job& job, int e_out) {
    return (job.flags & TMD_BP_DIRECTED) ? job.p - e_out : job.p + 1 - e_out;
}

const CoeffConsts& coeff_consts() {
    static const CoeffConsts* C = [] {
        CoeffConsts* c = new CoeffConsts();
        c->div.r[0] = fx::make_recip(1);
        for (int n = 1; n <= fx::SMALL_DIV_MAX; n++) c->div.r[n] = fx::make_recip((uint64_t)n);
        fx::Enc<LN2_LIMBS> e;
        fx::ln2_enc<LN2_LIMBS>(LN2_BITS, c->div, e);
        c->ln2_lo = e.lo;
        c->ln2_hi = e.hi;
        return c;
    }();
    return *C;
}

CoeffJob coeff_job(const tmd_job& job, int e_out) {
    CoeffJob J;
    J.func = job.func;
    J.e_in = job.e_in;
    J.p = job.p;
    J.d = job.d;
    J.L = (int)job.limbs;
    J.scale_log2 = scale_log2(job, e_out);
    J.log2_N = (int)job.log2_N;
    J.red = reduction_exponent(job.func, job.e_in, e_out);
    return J;
}

void host_anchor(const tmd_job& job, const std::vector<Segment>& segs, Anchor* A) {
    A->ok = 0;
    if (segs.empty()) return;
    uint64_t nb = 0, ns = 0;
    plan_counts(job, segs, &nb, &ns);
    if (nb < 2) return;
    job_anchor<ANCHOR_LIMBS>(coeff_job(job, segs[0].e_out), arg_mantissa(job, segs[0].j0), 64, coeff_consts(), *A);
}

tmd_status block_table(const tmd_job& job, const BlockPlan& blk, uint64_t* coeffs, uint64_t* table,
                       const Anchor* anchor) {
    const CoeffJob J = coeff_job(job, blk.e_out);
    const uint64_t M = arg_mantissa(job, blk.start);
    uint64_t c[(MAX_DEG + 1) * MAX_LIMBS];
    // Ziv: 512-bit words with 64 guard bits (from the anchor when there is
    // one), then 768-bit words with 320 computed directly
    if (!block_coeffs<8>(J, M, 64, coeff_consts(), c, anchor) && !block_coeffs<12>(J, M, 320, coeff_consts(), c))
        return TMD_EUNSUPPORTED;
    if (coeffs) coeffs_packed(J, c, coeffs);
    if (table) block_table_words(J, c, table);
    return TMD_OK;
}

// ------------------------------------------------------------ sound mode
// Upper bound of |f^(k)| over [x_lo, x_hi] (k >= 1 for log), in double with
// a relative margin.
static double deriv_max(int func, int k, double x_lo, double x_hi) {
    double v;
    if (func == TMD_EXP) {
        v = std::exp(x_hi);
    } else if (func == TMD_EXP2) {
        v = std::exp2(x_hi) * std::pow(std::log(2.0), (double)k);
    } else {
        double f = 1;
        for (int i = 2; i < k; i++) f *= i;  // (k-1)!
        v = k == 0 ? std::log(x_hi) : f / std::pow(x_lo, (double)k);
    }
    return v * (1.0 + 1e-9);
}

// eps_approx * 2^64 and eps_trunc * 2^64 for lines over `length` arguments
// (double precision, before the margins).
static tmd_status sound_bounds(const tmd_job& job, double length, double* ea_out, double* et_out, int* m_out,
                               uint32_t* log2_N) {
    tmd_job j = job;
    j.flags &= ~(uint32_t)TMD_SOUND;
    j.eps1 = j.eps3 = 0;
    tmd_status st = validate_job(j);
    if (st != TMD_OK) return st;
    std::vector<Segment> segs;
    st = plan_segments(j, segs);
    if (st != TMD_OK) return st;
    int e_min = segs[0].e_out;
    for (const Segment& s : segs) e_min = std::min(e_min, s.e_out);
    const int d = j.d, W = 64 * (int)j.limbs;
    const double u = std::ldexp(1.0, j.e_in - j.p);
    const double x_lo = std::ldexp((double)arg_mantissa(j, j.start), j.e_in - j.p);
    const double x_hi = std::ldexp((double)arg_mantissa(j, j.start + j.count - 1), j.e_in - j.p);
    const int s_log2 = scale_log2(j, e_min);
    const double T = std::ldexp(1.0, (int)j.log2_T), N = length > 0 ? length : std::ldexp(1.0, (int)j.log2_N);
    double fact[8] = {1, 1, 2, 6, 24, 120, 720, 5040};
    // eps_approx * 2^64: Taylor remainder plus coefficient rounding
    double ea = std::ldexp(std::pow(u * T, d + 1) * deriv_max(j.func, d + 1, x_lo, x_hi) / fact[d + 1],
                           s_log2 + 64);
    for (int k = 0; k <= d; k++) ea += std::ldexp(0.5 * std::pow(T, k), 64 - W);
    // eps_trunc * 2^64: dropped terms j >= 2 of the binomial expansion
    double cb[8];
    for (int k = 2; k <= d; k++)
        cb[k] = std::ldexp(std::pow(u, k) * deriv_max(j.func, k, x_lo, x_hi) / fact[k], s_log2 + W) + 0.5;
    double et = 0;
    for (int jj = 2; jj <= d; jj++) {
        double rj = 0;
        for (int k = jj; k <= d; k++) rj += cb[k] * fact[k] / fact[k - jj] * std::pow(T + d, k - jj);
        double binom = 1;
        for (int i = 0; i < jj; i++) binom *= (N - 1 - i) / (i + 1);
        et += rj * binom;
    }
    et = std::ldexp(et, 64 - W);
    const double margin = 1.0 + 1.0 / 1024;
    *ea_out = ea * margin + 4;
    *et_out = et * margin + 4;
    *m_out = j.m;
    *log2_N = j.log2_N;
    return TMD_OK;
}

tmd_status sound_eps(const tmd_job& job, uint64_t* eps1, uint64_t* eps3) {
    double ea, et;
    int m;
    uint32_t lN;
    tmd_status st = sound_bounds(job, 0, &ea, &et, &m, &lN);
    if (st != TMD_OK) return st;
    if (!(ea < 0x1p61) || !(et < 0x1p61)) return TMD_EINVAL;
    const uint64_t e3 = (1ull << (64 - m)) + (uint64_t)std::ceil(ea) + 1;
    const uint64_t e1 = e3 + (uint64_t)std::ceil(et) + (1ull << lN) + 2;
    if (e1 >= (1ull << 62)) return TMD_EINVAL;
    *eps1 = e1;
    *eps3 = e3;
    return TMD_OK;
}

uint32_t sound_piece_length(uint32_t log2_N) { return ((1u << log2_N) + 31u) / 32u; }

tmd_status sound_line_eps(const tmd_job& job, uint64_t eps3, uint64_t length, uint64_t* eps) {
    double ea, et;
    int m;
    uint32_t lN;
    if (length == 0 || length > (1ull << job.log2_N)) return TMD_EINVAL;
    tmd_status st = sound_bounds(job, (double)length, &ea, &et, &m, &lN);
    if (st != TMD_OK) return st;
    if (!(et < 0x1p61) || eps3 >= (1ull << 62)) return TMD_EINVAL;
    const uint64_t e = eps3 + (uint64_t)std::ceil(et) + length + 2;
    if (e >= (1ull << 62)) return TMD_EINVAL;
    *eps = e;
    return TMD_OK;
}

tmd_status sound_piece_eps(const tmd_job& job, uint64_t eps3, uint64_t* eps2) {
    return sound_line_eps(job, eps3, sound_piece_length(job.log2_N), eps2);
}

}  // namespace tmd
