// CUDA kernels of the hot path (sm_103a).
//
//   generation  Sect. IV-B/IV-C: each lane owns a packet of nu consecutive
//               sub-intervals of one Taylor block; it jumps to the packet's
//               first sub-interval with the straightforward shift (binomial
//               Toeplitz product of the block's difference column) and then
//               steps the tabulated differences with W-bit carry-chain adds.
//   search      Sect. III-B: Algorithm 4 (regular continued-fraction lower
//               bound, unrolled twice) on the 64-bit search words of each
//               line, one line per lane, the warp's 32 lines being
//               neighbouring sub-intervals; lines whose bound falls below
//               the threshold get their exact minimum and smallest argmin
//               from a Euclid-like recursion (exact_min) and are emitted by
//               warp ballot with one atomic per warp (Sect. III-C
//               compaction of failing sub-domains).  Lefevre's filter
//               (Algorithm 3) and the sound mode (eps'' filter, phase-2
//               pieces, phase 3 with its sub-pieces and the evaluation of
//               R_t at every argument of the failing ones) live in the
//               general kernel variant and in the line search only.
//
// Quotients: GB300 has no integer divide instruction and a slow FP64 unit,
// so floor(a/b) comes from an FP32 estimate built from 32-bit halves
// (I2F.U32 + FFMA), one reciprocal (MUFU) shared by both divisions of a
// half-step, and one integer correction.  With kf = fl(a) * rcp(fl(b)) the
// relative error is below 2^-21 (two round-toward-zero conversions of at most
// 2^-22 each after the FMA, 1 ulp for rcp.approx, half an ulp for the
// product), so for kf < 2^19 the estimate floor(max(kf - 1/2, 0)) is
// floor(a/b) or one less; one compare-and-subtract finishes it.  Larger
// quotients (rare: Gauss-Kuzmin tail) take an exact shift-subtract division.
#include <cuda_runtime.h>

#include "coeffs.cuh"
#include "dev.hpp"
#include "planrec.cuh"

namespace tmd {

#define FULLMASK 0xffffffffu

// ---------------------------------------------------------------- W-bit words
template <int L>
struct Word {
    uint64_t l[L];
};

template <int L>
__device__ __forceinline__ void w_add(Word<L>& a, const Word<L>& b) {
    if constexpr (L == 1) {
        a.l[0] += b.l[0];
    } else if constexpr (L == 2) {
        asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;"
            : "+l"(a.l[0]), "+l"(a.l[1])
            : "l"(b.l[0]), "l"(b.l[1]));
    } else {
        asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, %2, %5;"
            : "+l"(a.l[0]), "+l"(a.l[1]), "+l"(a.l[2])
            : "l"(b.l[0]), "l"(b.l[1]), "l"(b.l[2]));
    }
}

template <int L>
__device__ __forceinline__ void w_sub(Word<L>& a, const Word<L>& b) {
    if constexpr (L == 1) {
        a.l[0] -= b.l[0];
    } else if constexpr (L == 2) {
        asm("sub.cc.u64 %0, %0, %2;\n\tsubc.u64 %1, %1, %3;"
            : "+l"(a.l[0]), "+l"(a.l[1])
            : "l"(b.l[0]), "l"(b.l[1]));
    } else {
        asm("sub.cc.u64 %0, %0, %3;\n\tsubc.cc.u64 %1, %1, %4;\n\tsubc.u64 %2, %2, %5;"
            : "+l"(a.l[0]), "+l"(a.l[1]), "+l"(a.l[2])
            : "l"(b.l[0]), "l"(b.l[1]), "l"(b.l[2]));
    }
}

// a * c mod 2^W
template <int L>
__device__ __forceinline__ Word<L> w_mul_u64(const Word<L>& a, uint64_t c) {
    Word<L> r;
    uint64_t carry = 0;
#pragma unroll
    for (int i = 0; i < L; i++) {
        uint64_t lo = a.l[i] * c;
        uint64_t hi = __umul64hi(a.l[i], c);
        r.l[i] = lo + carry;
        carry = hi + (r.l[i] < lo ? 1ull : 0ull);
    }
    return r;
}

// acc += w * c mod 2^192 for a 32-bit c, on the six 32-bit words of the
// operands: the low halves of the six products c w_j go into one carry
// chain, the high halves (one word up) into a second.  SHIFT = 1 adds
// w * c * 2^32 instead (every product one word higher).
template <int SHIFT>
__device__ __forceinline__ void w3_madd32(Word<3>& acc, const Word<3>& w, uint32_t c) {
    uint32_t a[6], x[6];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        a[2 * i] = (uint32_t)acc.l[i];
        a[2 * i + 1] = (uint32_t)(acc.l[i] >> 32);
        x[2 * i] = (uint32_t)w.l[i];
        x[2 * i + 1] = (uint32_t)(w.l[i] >> 32);
    }
    if (SHIFT == 0) {
        asm("mad.lo.cc.u32 %0, %6, %12, %0;\n\t"
            "madc.lo.cc.u32 %1, %7, %12, %1;\n\t"
            "madc.lo.cc.u32 %2, %8, %12, %2;\n\t"
            "madc.lo.cc.u32 %3, %9, %12, %3;\n\t"
            "madc.lo.cc.u32 %4, %10, %12, %4;\n\t"
            "madc.lo.u32 %5, %11, %12, %5;\n\t"
            "mad.hi.cc.u32 %1, %6, %12, %1;\n\t"
            "madc.hi.cc.u32 %2, %7, %12, %2;\n\t"
            "madc.hi.cc.u32 %3, %8, %12, %3;\n\t"
            "madc.hi.cc.u32 %4, %9, %12, %4;\n\t"
            "madc.hi.u32 %5, %10, %12, %5;"
            : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5])
            : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(c));
    } else {
        asm("mad.lo.cc.u32 %1, %6, %12, %1;\n\t"
            "madc.lo.cc.u32 %2, %7, %12, %2;\n\t"
            "madc.lo.cc.u32 %3, %8, %12, %3;\n\t"
            "madc.lo.cc.u32 %4, %9, %12, %4;\n\t"
            "madc.lo.u32 %5, %10, %12, %5;\n\t"
            "mad.hi.cc.u32 %2, %6, %12, %2;\n\t"
            "madc.hi.cc.u32 %3, %7, %12, %3;\n\t"
            "madc.hi.cc.u32 %4, %8, %12, %4;\n\t"
            "madc.hi.u32 %5, %9, %12, %5;"
            : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5])
            : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(c));
    }
#pragma unroll
    for (int i = 0; i < 3; i++) acc.l[i] = ((uint64_t)a[2 * i + 1] << 32) | a[2 * i];
}

// acc += w * binom(i0, J) mod 2^W in the straightforward shift, i0 < 2^16:
// binom(i0, 1) and binom(i0, 2) are below 2^32 and binom(i0, 3) below 2^46,
// so for 192-bit words the product takes one or two 32-bit multiplier
// passes instead of a full 64 x 64-bit product per limb.
template <int L, int J>
__device__ __forceinline__ void w_madd_binom(Word<L>& acc, const Word<L>& w, uint64_t c) {
    if constexpr (L == 3 && J <= 2) {
        w3_madd32<0>(acc, w, (uint32_t)c);
    } else if constexpr (L == 3 && J == 3) {
        w3_madd32<0>(acc, w, (uint32_t)c);
        w3_madd32<1>(acc, w, (uint32_t)(c >> 32));
    } else {
        w_add<L>(acc, w_mul_u64<L>(w, c));
    }
}

// binom(n, j), j = 0..4, exact for n <= 2^16
__device__ __forceinline__ void binomials(uint64_t n, uint64_t* c) {
    c[0] = 1;
    c[1] = n;
    c[2] = n * (n - 1) / 2;
    c[3] = c[2] * (n - 2) / 3;
    c[4] = c[3] * (n - 3) / 4;
}

// ------------------------------------------------------------------ quotients
__device__ __forceinline__ float u64_to_f32_rz(uint64_t x) {
    return __fmaf_rz(__uint2float_rz((uint32_t)(x >> 32)), 4294967296.0f,
                     __uint2float_rz((uint32_t)x));
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Quotient estimate.  af = fl(a) and bf = fl(b) come from u64_to_f32_rz
// (a (1 - 2^-22) <= af <= a), rbs = fl(rcp(bf) (1 - 2^-20)) carries a
// deliberate downward bias, kf = fl(af rbs).  With 1 ulp for rcp.approx and
// half an ulp for each product,
//     (a/b)(1 - 1.5 2^-20) <= kf <= (a/b)(1 - 2^-21) < a/b,
// so for kf < 2^19: floor(a/b) - 1 <= floor(kf) <= floor(a/b).  floor(kf) is
// read off the bits of 2^23 + kf rounded toward zero.  *ok is false when the
// estimate is outside the fast range (the caller then divides exactly).
__device__ __forceinline__ uint32_t quot_estimate(float af, float rbs, bool& ok) {
    const float kf = af * rbs;
    ok = kf < 524288.0f;  // 2^19
    return __float_as_uint(__fadd_rz(kf, 8388608.0f)) - 0x4B000000u;
}

__device__ __forceinline__ float scaled_rcp(float bf) {
    return rcp_approx(bf) * 0.99999904632568359375f;  // 1 - 2^-20
}

// x >= b ? x - b : x on 64-bit words without a compare and select: the
// borrow of x - b, as a 0 / all-ones mask, adds b back (the subtract-with-
// borrow and add-with-carry chains issue at the full 32-bit add rate, the
// compares and selects they replace on the half-rate logic pipe).
__device__ __forceinline__ uint64_t csub(uint64_t x, uint64_t b, uint32_t& bw) {
    uint32_t t0, t1;
    asm("sub.cc.u32 %0, %3, %5;\n\tsubc.cc.u32 %1, %4, %6;\n\tsubc.u32 %2, 0, 0;"
        : "=r"(t0), "=r"(t1), "=r"(bw)
        : "r"((uint32_t)x), "r"((uint32_t)(x >> 32)), "r"((uint32_t)b), "r"((uint32_t)(b >> 32)));
    asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, %3;"
        : "+r"(t0), "+r"(t1)
        : "r"((uint32_t)b & bw), "r"((uint32_t)(b >> 32) & bw));
    return ((uint64_t)t1 << 32) | t0;
}

__device__ __forceinline__ uint64_t csub(uint64_t x, uint64_t b) {
    uint32_t bw;
    return csub(x, b, bw);
}

// r = a - k b for an estimate k in {floor(a/b) - 1, floor(a/b)}, then one
// conditional subtract; k is raised when the subtract happens (its borrow
// mask is 0 then, all ones otherwise: k + 1 + mask).
__device__ __forceinline__ uint64_t rem_fix(uint64_t a, uint64_t b, uint32_t& k) {
    const uint64_t r = a - (uint64_t)k * b;
    uint32_t bw;
    const uint64_t rr = csub(r, b, bw);
    k += 1u + bw;
    return rr;
}

// exact floor(a/b), a mod b (b > 0) by shift-subtract; the quotient is
// returned clamped to 2^20 (it only feeds the saturating u/v update)
__device__ __noinline__ uint64_t divmod_slow(uint64_t a, uint64_t b, uint32_t& k) {
    uint64_t quo = 0, rem = 0;
    int top = a ? 63 - __clzll((long long)a) : -1;
    for (int i = top; i >= 0; i--) {
        bool hi = (rem >> 63) != 0;
        rem = (rem << 1) | ((a >> i) & 1ull);
        if (hi || rem >= b) {
            rem -= b;
            quo |= 1ull << i;
        }
    }
    k = quo < (1ull << 20) ? (uint32_t)quo : (1u << 20);
    return rem;
}

__device__ __forceinline__ uint32_t sat_madd(uint32_t u, uint32_t k, uint32_t v, uint32_t n) {
    const uint32_t kc = min(k, n);
    const uint32_t s = u + kc * v;  // u, v < n <= 2^16, kc <= 2^16: no wrap
    return min(s, n);
}

// General half-step by FP32 estimates: k = floor(a/b) (a > b > 0),
// a' = a mod b, and the reduction of x modulo b.  X_BELOW: x < a is known
// (inside the loop d stays below the dividend), so x's estimate is in the
// fast range whenever a's is (the estimate is monotonic in the dividend)
// and only a's range is checked.
template <bool X_BELOW>
__device__ __forceinline__ void half_step_div(uint64_t a, uint64_t b, uint64_t x, uint64_t& a_out,
                                              uint32_t& k_out, uint64_t& x_out) {
    const float rbs = scaled_rcp(u64_to_f32_rz(b));
    bool ok1, ok2;
    uint32_t k = quot_estimate(u64_to_f32_rz(a), rbs, ok1);
    uint32_t kx = quot_estimate(u64_to_f32_rz(x), rbs, ok2);
    uint64_t an = rem_fix(a, b, k);
    uint64_t xn = rem_fix(x, b, kx);
    if (!(ok1 && (X_BELOW || ok2))) {
        an = divmod_slow(a, b, k);
        xn = divmod_slow(x, b, kx);
    }
    a_out = an;
    k_out = k;
    x_out = xn;
}

// Second half-step by FP32 estimates: k = floor(p/q), p' = p mod q, then
// d <- (d - p') mod q when d >= p' (d - p' < k q <= p: its estimate is in
// the fast range whenever p's is, so only p's range is checked).
__device__ __forceinline__ void second_half_div(uint64_t& p, uint64_t q, uint64_t& d, uint32_t& k) {
    const float rqs = scaled_rcp(u64_to_f32_rz(q));
    bool ok1, ok2;
    uint32_t kk = quot_estimate(u64_to_f32_rz(p), rqs, ok1);
    uint64_t pn = rem_fix(p, q, kk);
    bool ge = d >= pn;
    uint64_t e = ge ? d - pn : 0ull;
    uint32_t ke = quot_estimate(u64_to_f32_rz(e), rqs, ok2);
    uint64_t en = rem_fix(e, q, ke);
    (void)ok2;
    if (!ok1) {
        pn = divmod_slow(p, q, kk);
        ge = d >= pn;
        en = divmod_slow(ge ? d - pn : 0ull, q, ke);
    }
    d = ge ? en : d;
    p = pn;
    k = kk;
}

// Algorithm 4 lower bound of min_{0<=x<n} (B - A x) mod 2^64 on integers
// scaled by 2^64: p <- A, q <- 2^64, d <- B, u <- 1, v <- 0; returns d when
// u + v >= n.  Endings of a rational expansion: p = 0 -> d mod q (already
// reduced), q = 0 -> d.  *hs counts half-steps.
//
// The dividend of every half-step exceeds its divisor (q mod p < p and
// p mod q < q), so the partial quotient is k >= 1, and k = 1 exactly when
// a - b < b.  That case -- 41.5 % of partial quotients (Gauss-Kuzmin) -- is
// done by subtraction alone: the reduced value is below 2b there, so one
// compare-and-subtract reduces it (the hybrid subtractive/division scheme of
// Sect. III-A).  Neighbouring lines share their partial quotients, so the
// branch is nearly always uniform across a warp.
__device__ __forceinline__ uint64_t cf_lower_bound(uint64_t B, uint64_t A, uint32_t n, uint32_t* hs) {
    if (A == 0) {
        *hs = 0;
        return B;
    }
    uint64_t p = A, q, d = B;
    uint32_t u = 1, v = 0, h = 1;
    // first half-step with q = 2^64: floor(2^64/p) = floor((2^64 - p)/p) + 1,
    // and u = 1 + k * 0 stays 1
    {
        uint32_t k;
        half_step_div<false>(0ull - p, p, d, q, k, d);
    }
    if (1u >= n || q == 0) {
        *hs = h;
        return d;
    }
#pragma unroll 1
    for (int guard = 0; guard < 64; guard++) {
        // second half: k = floor(p/q); p -= k q; v += k u; if d >= p: d = (d - p) mod q
        {
            const uint64_t r = p - q;
            if (r < q) {
                p = r;
                v = min(v + u, n);
                d = csub(d, p);  // d - p < k q = q
            } else {
                uint32_t k;
                second_half_div(p, q, d, k);
                v = sat_madd(v, k, u, n);
            }
            h++;
            // exit at u + v >= n, or when p reached 0 (d was reduced mod q
            // just above): one branch for both
            if ((u + v >= n) | (p == 0)) break;
        }
        // first half: k = floor(q/p); q -= k p; u += k v; d = d mod p
        {
            const uint64_t r = q - p;
            if (r < p) {
                q = r;
                u = min(u + v, n);
                d = csub(d, p);  // d < q < 2p
            } else {
                uint32_t k;
                half_step_div<true>(q, p, d, q, k, d);
                u = sat_madd(u, k, v, n);
            }
            h++;
            if ((u + v >= n) | (q == 0)) break;
        }
    }
    *hs = h;
    return d;
}

__device__ __forceinline__ uint64_t udivmod64(uint64_t x, uint64_t b, uint64_t* r);

// ------------------------------------------------ Lefevre, Algorithm 3
// k = floor(a / b) clamped to 2^20 (it only feeds the saturating counts) and
// a mod b, for any a and b > 0: no division for k <= 1, else an FP32
// estimate and one correction, else (k >= 2^19) the exact slow division.
__device__ __forceinline__ uint64_t quot_rem(uint64_t a, uint64_t b, uint32_t& k) {
    if (a < b) {
        k = 0;
        return a;
    }
    const uint64_t r1 = a - b;
    if (r1 < b) {
        k = 1;
        return r1;
    }
    bool ok;
    k = quot_estimate(u64_to_f32_rz(a), scaled_rcp(u64_to_f32_rz(b)), ok);
    uint64_t r = rem_fix(a, b, k);
    if (!ok) r = divmod_slow(a, b, k);
    return r;
}

// Lefevre's lower bound (Algorithm 3, the swap form of Algorithm 1) of
// min_{0<=x<n} (B - A x) mod 2^64: p <- A, q <- 2^64 - A, d <- B, u <- v <- 1.
// Each iteration moves d to the point just added at its left when b is on
// the swapped side (d -= l, l = Algorithm 1's p, held in q after a swap),
// takes a whole quotient k = floor(q/p) off q (u += k v), the first unit of
// the next one off p (v += u), and swaps (p, q), (u, v) when b changes side.
// Returns d at the first u + v >= n; a division leaving a zero remainder
// ends the loop with d reduced modulo the other length (rational a).
// *iters = loop iterations (Table 3).  u, v saturate at n.
// SPEC: Lefevre's specific instructions, read as taking a run of
// consecutive iterations with quotient 0 in one iteration by exact
// divisions: on the swapped side (q < p here: each d -= q, p -= q, v += u)
// r = min(floor(d/q), floor((p-1)/q), the iterations left before u + v >= n);
// on the other (q < p: each p -= q, v += u) r = ceil((p - max(d, q))/q) or
// fewer if u + v reaches n.  Same states, far fewer iterations.
template <bool SPEC>
__device__ __noinline__ uint64_t lefevre_lower_bound(uint64_t B, uint64_t A, uint32_t n, uint32_t* iters) {
    if (A == 0) {
        *iters = 0;
        return B;
    }
    uint64_t p = A, q = 0ull - A, d = B;
    uint32_t u = 1, v = 1, it = 0;
    bool sw = false;
    if (d >= p) {
        const uint64_t t = p;
        p = q;
        q = t;
        sw = true;
    }
#pragma unroll 1
    for (; it < (1u << 17); ) {  // u + v grows by at least one per iteration
        it++;
        if (SPEC && !sw && q < p) {
            // a run of unswapped iterations with quotient 0 (d < p, q < p:
            // each p -= q, v += u while p stays above d and q)
            uint64_t rem;
            const uint64_t big = d > q ? d : q;
            const uint64_t r = udivmod64(p - big - 1, q, &rem) + 1;
            const uint64_t jx = u + v >= n ? 1ull : (uint64_t)((n - v + u - 1) / u);
            if (jx <= r) break;  // d is unchanged by the run
            p -= r * q;
            v += (uint32_t)r * u;  // < n
        } else if (SPEC && sw && q < p) {
            uint64_t rem;
            const uint64_t rd = udivmod64(d, q, &rem);
            const uint64_t rp = udivmod64(p - 1, q, &rem);
            // iterations up to the one whose exit test fires: the least j >= 1
            // with v + j u >= n (u >= 1; v <= n)
            const uint64_t jx = v + u >= n ? 1ull : (uint64_t)((n - v + u - 1) / u);
            const uint64_t r = min(min(rd, rp), jx);
            d -= r * q;
            if ((uint64_t)v + r * (uint64_t)u >= (uint64_t)n) break;
            p -= r * q;
            v += (uint32_t)r * u;  // < n
        } else {
            if (sw) d -= q;
            uint32_t k;
            q = quot_rem(q, p, k);
            u = sat_madd(u, k, v, n);
            if (u + v >= n) break;
            if (q == 0) {
                uint32_t kk;
                d = quot_rem(d, p, kk);
                break;
            }
            p -= q;
            v = min(v + u, n);
        }
        const uint64_t l = sw ? q : p;
        if (sw != (d >= l)) {
            const uint64_t t = p;
            p = q;
            q = t;
            const uint32_t w = u;
            u = v;
            v = w;
            sw = !sw;
        }
    }
    *iters = it;
    return d;
}

// -------------------------------------------------------------- compaction
__device__ __forceinline__ void emit_warp(bool has, uint32_t job, uint32_t sub, uint64_t arg,
                                          uint64_t val, tmd_candidate* cand, uint64_t cap,
                                          uint64_t* count) {
    unsigned mask = __ballot_sync(FULLMASK, has);
    if (mask == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd((unsigned long long*)count, (unsigned long long)__popc(mask));
    base = __shfl_sync(FULLMASK, base, leader);
    if (has) {
        uint64_t idx = base + (uint64_t)__popc(mask & ((1u << lane) - 1u));
        if (idx < cap) {
            tmd_candidate c;
            c.job = job;
            c.subint = sub;
            c.arg_index = arg;
            c.value = val;
            cand[idx] = c;
        }
    }
}

// ------------------------------------------------------- exact minimum
// floor(x / b) for any b > 0: FP32 estimates that never exceed the quotient
// (round-toward-zero conversions, a reciprocal biased down by 2^-20), each
// removing ~20 bits of it, then compare-and-subtract; *r = x mod b.
__device__ __forceinline__ uint64_t udivmod64(uint64_t x, uint64_t b, uint64_t* r) {
    const float rb = scaled_rcp(u64_to_f32_rz(b));
    uint64_t q = 0;
#pragma unroll 1
    for (int it = 0; it < 6 && x >= b; it++) {
        const float kf = u64_to_f32_rz(x) * rb;  // <= x / b
        uint64_t t;
        if (kf < 4194304.0f)
            t = (uint64_t)(__float_as_uint(__fadd_rz(kf, 8388608.0f)) - 0x4B000000u);
        else
            t = __float2ull_rz(kf);
        if (t == 0) t = 1;  // x >= b here, so floor(x / b) >= 1
        x -= t * b;
        q += t;
    }
    if (x >= b) {  // not reached for b >= 1 (each pass leaves x < 2^-19 x + 2b)
        uint32_t k;
        x = divmod_slow(x, b, k);
        q = ~0ull;
    }
    *r = x;
    return q;
}

// floor((hi 2^64 + lo) / m) for a quotient known to be below 2^16 (m > 0).
__device__ __forceinline__ uint64_t udiv128_small(uint64_t hi, uint64_t lo, uint64_t m) {
    const float nf = __fmaf_rz((float)hi, 18446744073709551616.0f, u64_to_f32_rz(lo));  // <= value
    const float kf = nf * scaled_rcp(u64_to_f32_rz(m));                               // <= quotient
    uint64_t t = (uint64_t)(__float_as_uint(__fadd_rz(kf, 8388608.0f)) - 0x4B000000u);
    // remainder (hi:lo) - t m, then at most a few compare-and-subtracts
    uint64_t plo = t * m, phi = __umul64hi(t, m);
    uint64_t rlo = lo - plo, rhi = hi - phi - (lo < plo ? 1ull : 0ull);
#pragma unroll 1
    for (int it = 0; it < 4 && (rhi != 0 || rlo >= m); it++) {
        rhi -= rlo < m ? 1ull : 0ull;
        rlo -= m;
        t++;
    }
    return t;
}

// Exact min_{0<=x<n} (B - A x) mod 2^64 and its smallest argmin (n >= 1),
// without visiting the n points.  The sequence y_x = (b - c x) mod m falls
// by c until it wraps, so only the ends of its runs and its last point can
// be minima; the value at the end of run w is (b + w m) mod c -- a rising
// sequence modulo c.  A rising sequence (b + a x) mod m can only have its
// minimum at x = 0 or just after a wrap, and the value after wrap k is
// (b - k m) mod a -- a falling sequence modulo a.  Each form hands the next
// the same candidate values on a smaller modulus (m, c) -> (c, m mod c), the
// Euclidean algorithm, with fewer points; a running minimum of the direct
// candidates is the answer.  The smallest argmin then follows from
// A x = B - min (mod 2^64): with A = 2^t A', x = ((B - min) / 2^t) A'^-1
// mod 2^(64-t), the least solution, which lies below n.
__device__ __noinline__ uint64_t exact_min(uint64_t B, uint64_t A, uint32_t n, uint32_t* argmin) {
    if (A == 0 || n <= 1) {
        *argmin = 0;
        return B;
    }
    // level 0, falling form with modulus 2^64: runs end where the subtraction wraps
    uint64_t best;
    uint64_t m, c, b, cnt;
    {
        const uint64_t Tl = A * (uint64_t)(n - 1), Th = __umul64hi(A, (uint64_t)(n - 1));
        best = B - Tl;  // last point
        uint64_t W = 0;
        if (Th != 0 || Tl > B) {  // W = ceil((T - B) / 2^64)
            const uint64_t dl = Tl - B, dh = Th - (Tl < B ? 1ull : 0ull);
            W = dh + (dl != 0 ? 1ull : 0ull);
        }
        cnt = W;
        if (cnt) {
            // rising form: (B mod A + w (2^64 mod A)) mod A, w < W
            uint64_t bm, mm;
            udivmod64(B, A, &bm);
            udivmod64(0ull - A, A, &mm);  // 2^64 mod A = (2^64 - A) mod A
            m = A;
            c = mm;
            b = bm;
        }
    }
    bool rising = true;
#pragma unroll 1
    for (int level = 0; level < 200 && cnt != 0; level++) {
        if (rising) {
            // (b + a x) mod m, x < cnt, a = c: minimum at x = 0 or after a wrap
            best = b < best ? b : best;
            const uint64_t a = c;
            if (a == 0) break;
            // K = floor((b + a (cnt - 1)) / m) wraps
            uint64_t lo = a * (cnt - 1), hi = __umul64hi(a, cnt - 1);
            lo += b;
            hi += lo < b ? 1ull : 0ull;
            const uint64_t K = udiv128_small(hi, lo, m);
            if (K == 0) break;
            // after wrap k: (b - k m) mod a = (b mod a - (k mod ...) ) -> falling form
            uint64_t bm, mm;
            udivmod64(b, a, &bm);
            udivmod64(m, a, &mm);
            const uint64_t b2 = bm >= mm ? bm - mm : bm + (a - mm);  // (b - m) mod a
            cnt = K;
            m = a;
            c = mm;
            b = b2;
            rising = false;
        } else {
            // (b - c x) mod m, x < cnt: minimum at the end of a run or at the last point
            if (c == 0) {
                best = b < best ? b : best;
                break;
            }
            const uint64_t Tl = c * (cnt - 1), Th = __umul64hi(c, cnt - 1);
            uint64_t W = 0;
            if (Th != 0 || Tl > b) {  // W = ceil((T - b) / m) = floor((T - b - 1) / m) + 1
                uint64_t dl = Tl - b, dh = Th - (Tl < b ? 1ull : 0ull);
                dh -= dl == 0 ? 1ull : 0ull;
                dl -= 1;
                W = udiv128_small(dh, dl, m) + 1;
            }
            const uint64_t last = b + W * m - Tl;  // exact, below m
            best = last < best ? last : best;
            if (W == 0) break;
            uint64_t bm, mm;
            udivmod64(b, c, &bm);
            udivmod64(m, c, &mm);
            cnt = W;
            m = c;
            c = mm;
            b = bm;
            rising = true;
        }
    }
    // least x with A x = B - best (mod 2^64)
    const int t = __ffsll((long long)A) - 1;
    const uint64_t ao = A >> t;
    uint64_t inv = ao;  // correct to 3 bits; each Newton step doubles that
#pragma unroll
    for (int i = 0; i < 5; i++) inv *= 2ull - ao * inv;
    uint64_t x = ((B - best) >> t) * inv;
    if (t > 0) x &= (~0ull) >> t;
    *argmin = (uint32_t)x;
    return best;
}

// Exact resolution of the flagged lines of a warp, then compaction.  Each
// flagged lane finds its line's minimum and smallest argmin by exact_min;
// in all-hits mode every argument of each flagged line is visited by the
// whole warp (x = lane, lane + 32, ...) and every one below the threshold
// is reported.
__device__ __noinline__ void resolve_and_emit(bool fail, uint64_t B, uint64_t A, uint32_t n,
                                              uint64_t Tm, bool all_hits, uint32_t job,
                                              uint32_t sub, uint64_t arg_base,
                                              tmd_candidate* cand, uint64_t cap, uint64_t* count) {
    if (!all_hits) {
        uint64_t mn = 0;
        uint32_t x = 0;
        if (fail) mn = exact_min(B, A, n, &x);
        emit_warp(fail && mn < Tm, job, sub, arg_base + x, mn, cand, cap, count);
        return;
    }
    const int lane = threadIdx.x & 31;
    unsigned fails = __ballot_sync(FULLMASK, fail);
    while (fails) {
        const int src = __ffs(fails) - 1;
        fails &= fails - 1u;
        const uint64_t Bs = __shfl_sync(FULLMASK, B, src);
        const uint64_t As = __shfl_sync(FULLMASK, A, src);
        const uint32_t ns = __shfl_sync(FULLMASK, n, src);
        const uint32_t js = __shfl_sync(FULLMASK, job, src);
        const uint32_t ss = __shfl_sync(FULLMASK, sub, src);
        const uint64_t ab = __shfl_sync(FULLMASK, arg_base, src);
        uint64_t val = Bs - As * (uint64_t)lane;
        const uint64_t step = As * 32ull;
        const uint32_t trips = (ns + 31u) >> 5;
        for (uint32_t t = 0; t < trips; t++) {
            const uint32_t x = t * 32u + (uint32_t)lane;
            emit_warp(x < ns && val < Tm, js, ss, ab + x, val, cand, cap, count);
            val -= step;
        }
    }
}

__device__ __forceinline__ void flush_stats(uint64_t* stats, uint32_t lines, uint32_t fail, uint32_t half) {
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        lines += __shfl_xor_sync(FULLMASK, lines, off);
        fail += __shfl_xor_sync(FULLMASK, fail, off);
        half += __shfl_xor_sync(FULLMASK, half, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd((unsigned long long*)&stats[ST_LINES], (unsigned long long)lines);
        atomicAdd((unsigned long long*)&stats[ST_FAIL], (unsigned long long)fail);
        atomicAdd((unsigned long long*)&stats[ST_HALF], (unsigned long long)half);
    }
}

// ---------------------------------------------------------- packet machinery
template <int L, int D>
struct Packet {
    Word<L> d0[D + 1];  // Delta^l g0 at the current sub-interval, l = 0..D
    Word<L> d1[D];      // Delta^l g1, l = 0..D-1
    DevBlock blk;
    uint32_t i0, i1;    // sub-interval range of the packet within the block
    bool active;
};

// Delta^l <- sum_{k>=l} binom(i0, k-l) Delta^k(0), l = 0..E, in place
// (ascending l only reads the still-unshifted higher orders); E is the
// column's top order.
template <int L, int E, int l, int k>
__device__ __forceinline__ void shift_terms(Word<L>* col, const uint64_t* c) {
    if constexpr (k <= E) {
        w_madd_binom<L, k - l>(col[l], col[k], c[k - l]);
        shift_terms<L, E, l, k + 1>(col, c);
    }
}

template <int L, int E, int l>
__device__ __forceinline__ void shift_column(Word<L>* col, const uint64_t* c) {
    if constexpr (l < E) {
        shift_terms<L, E, l, l + 1>(col, c);
        shift_column<L, E, l + 1>(col, c);
    }
}

template <int L, int D>
__device__ __forceinline__ uint32_t packet_init(Packet<L, D>& P, const DevTask& t, const DevJob& job,
                                                const LaunchArgs& a) {
    const int lane = threadIdx.x & 31;
    P.active = (uint32_t)lane < t.count;
    const uint64_t g = t.g0 + (P.active ? (uint64_t)lane : 0ull);
    // the packet's block from the job's segment table: within a segment
    // every block but the last holds ppb packets (the block records' own
    // formula, planrec.cuh), so no search over the block records is needed
    // (segment fields read from the job record in global memory: indexing a
    // register copy by the segment number would move it to local memory)
    const DevJob& jg = a.jobs[t.job];
    const uint64_t rp = g - job.packet_off;
    uint32_t sg = 0;
    for (uint32_t k = 1; k < job.n_seg; k++)
        if (jg.seg_packet0[k] <= rp) sg = k;
    const uint32_t bis = (uint32_t)(rp - jg.seg_packet0[sg]) / job.ppb;
    const uint32_t lo = job.block_off + (uint32_t)jg.seg_block0[sg] + bis;
    P.blk = a.blocks[lo];
    const uint64_t pk = g - P.blk.packet_off;
    P.i0 = (uint32_t)(pk * job.nu);
    P.i1 = min(P.i0 + job.nu, P.blk.n_sub);
    const uint64_t* tw = a.tables + P.blk.table_off;
#pragma unroll
    for (int w = 0; w <= D; w++)
#pragma unroll
        for (int l = 0; l < L; l++) P.d0[w].l[l] = __ldg(tw + w * L + l);
#pragma unroll
    for (int w = 0; w < D; w++)
#pragma unroll
        for (int l = 0; l < L; l++) P.d1[w].l[l] = __ldg(tw + (D + 1 + w) * L + l);
    // straightforward shift to sub-interval i0, in place (ascending l only
    // reads the still-unshifted higher orders):
    // Delta^l(i0) = sum_{k>=l} binom(i0, k-l) Delta^k(0)
    uint64_t c[5];
    binomials(P.i0, c);
    shift_column<L, D, 0>(P.d0, c);
    shift_column<L, D - 1, 0>(P.d1, c);
    return lo;
}

// one tabulated-difference step: Delta^l(i+1) = Delta^l(i) + Delta^(l+1)(i), l ascending
template <int L, int D>
__device__ __forceinline__ void packet_step(Packet<L, D>& P) {
#pragma unroll
    for (int l = 0; l < D; l++) w_add<L>(P.d0[l], P.d0[l + 1]);
#pragma unroll
    for (int l = 0; l + 1 < D; l++) w_add<L>(P.d1[l], P.d1[l + 1]);
}

// search words of the current line (top limb of b plus the shift -- 2^(64-m),
// or eps1 in sound mode --, top limb of -alpha)
template <int L, int D>
__device__ __forceinline__ void packet_words(const Packet<L, D>& P, uint64_t shift, uint64_t& B, uint64_t& A) {
    B = P.d0[0].l[L - 1] + shift;
    uint64_t low = 0;
#pragma unroll
    for (int l = 0; l + 1 < L; l++) low |= P.d1[0].l[l];
    A = ~P.d1[0].l[L - 1] + (low == 0 ? 1ull : 0ull);
}

// R_t(y) mod 2^W by Horner from the block's Taylor coefficients.
template <int L, int D>
__device__ __forceinline__ Word<L> poly_at(const Word<L>* c, uint64_t y) {
    Word<L> acc = c[D];
#pragma unroll
    for (int k = D - 1; k >= 0; k--) {
        acc = w_mul_u64<L>(acc, y);
        w_add<L>(acc, c[k]);
    }
    return acc;
}

// Sound mode after the filter (Sect. III-A phases 2 and 3).  A line of the
// warp that failed Algorithm 4 and whose exact minimum is below 2 eps1 is
// cut into 32 pieces of n2 = ceil(N/32) arguments, one per lane; each lane
// forms its piece's own line from the block polynomial (R_t at the piece
// start and the next argument, the search words shifted by eps2) and keeps
// the piece if its exact minimum is below 2 eps2 (phase 2; Algorithm 4's
// bound clears most pieces before the exact minimum is formed).  Phase 3 takes
// the kept pieces one at a time with the whole warp.  A piece of more than
// 64 arguments is first cut the same way into 32 sub-pieces of
// ceil(n2/32) arguments, tested against their own half-width eps2s, and R_t
// is evaluated by Horner at every argument of the failing sub-pieces; a
// shorter piece has R_t evaluated at each of its arguments directly, lane l
// starting at the piece start + l with the step-32 forward differences of
// R_t (Horner at y0, y0 + 32, ..., y0 + 32 D) and stepping them.  Every
// argument with (top64(R_t(y)) + eps3) mod 2^64 < 2 eps3 is emitted.
template <int L>
__device__ __forceinline__ bool piece_line_fails(const Word<L>& r0, Word<L> r1, uint64_t shift, uint64_t T,
                                                 uint32_t len) {
    w_sub<L>(r1, r0);
    uint64_t low = 0;
#pragma unroll
    for (int l = 0; l + 1 < L; l++) low |= r1.l[l];
    const uint64_t B = r0.l[L - 1] + shift;
    const uint64_t A = ~r1.l[L - 1] + (low == 0 ? 1ull : 0ull);
    // Algorithm 4's lower bound first: a piece whose bound reaches T cannot
    // come within it (most pieces; the exact minimum costs several 64-bit
    // divisions per level), the others are decided exactly
    uint32_t hs;
    if (cf_lower_bound(B, A, len, &hs) >= T) return false;
    uint32_t xm;
    return exact_min(B, A, len, &xm) < T;
}

template <int L, int D>
__device__ __noinline__ void sound_exhaustive(bool fail, uint64_t B, uint64_t A, uint32_t n, uint64_t table_off,
                                              uint32_t i, uint32_t sub, uint64_t arg_base, uint32_t job,
                                              const DevJob& jb, const LaunchArgs& a) {
    const int lane = threadIdx.x & 31;
    bool go = false;
    if (fail) {
        uint32_t xm;
        go = exact_min(B, A, n, &xm) < jb.Tm;
    }
    const uint32_t n2 = ((1u << jb.log2_N) + 31u) >> 5;
    const uint32_t n3 = (n2 + 31u) >> 5;
    const bool two_level = jb.T2s != 0;
    uint32_t exh = 0, refined = 0;  // identical on every lane
    unsigned todo = __ballot_sync(FULLMASK, go);
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1u;
        const uint64_t toff = __shfl_sync(FULLMASK, table_off, src);
        const uint32_t is = __shfl_sync(FULLMASK, i, src);
        const uint32_t ns = __shfl_sync(FULLMASK, n, src);
        const uint32_t ss = __shfl_sync(FULLMASK, sub, src);
        const uint64_t ab = __shfl_sync(FULLMASK, arg_base, src);
        const uint32_t js = __shfl_sync(FULLMASK, job, src);
        const uint64_t* cw = a.tables + toff + (2 * D + 1) * L;
        Word<L> c[D + 1];
#pragma unroll
        for (int k = 0; k <= D; k++)
#pragma unroll
            for (int l = 0; l < L; l++) c[k].l[l] = __ldg(cw + k * L + l);
        const uint64_t ybase = (uint64_t)is << jb.log2_N;
        // phase 2: this lane's piece [x0, x0 + len)
        const uint32_t x0 = (uint32_t)lane * n2;
        const uint32_t len = x0 < ns ? min(n2, ns - x0) : 0u;
        bool keep = false;
        if (len)
            keep = piece_line_fails<L>(poly_at<L, D>(c, ybase + x0), poly_at<L, D>(c, ybase + x0 + 1), jb.shift2,
                                       jb.T2, len);
        unsigned pieces = __ballot_sync(FULLMASK, keep);
        while (pieces) {
            const uint32_t pc = (uint32_t)(__ffs(pieces) - 1);
            pieces &= pieces - 1u;
            const uint32_t px0 = pc * n2;
            const uint32_t pend = min(px0 + n2, ns);
            refined += pend - px0;
            if (two_level) {
                // this lane's sub-piece [s0, s0 + slen) of the piece
                const uint32_t s0 = px0 + (uint32_t)lane * n3;
                const uint32_t slen = s0 < pend ? min(n3, pend - s0) : 0u;
                bool keep2 = false;
                if (slen)
                    keep2 = piece_line_fails<L>(poly_at<L, D>(c, ybase + s0), poly_at<L, D>(c, ybase + s0 + 1),
                                                jb.shift2s, jb.T2s, slen);
                unsigned subs = __ballot_sync(FULLMASK, keep2);
                while (subs) {
                    const uint32_t sp = (uint32_t)(__ffs(subs) - 1);
                    subs &= subs - 1u;
                    const uint32_t sx0 = px0 + sp * n3;
                    const uint32_t send = min(sx0 + n3, pend);
                    exh += send - sx0;
                    const uint32_t trips = (send - sx0 + 31u) >> 5;
#pragma unroll 1
                    for (uint32_t t = 0; t < trips; t++) {
                        const uint32_t x = sx0 + t * 32u + (uint32_t)lane;
                        const uint64_t val = poly_at<L, D>(c, ybase + x).l[L - 1] + jb.shift3;
                        emit_warp(x < send && val < jb.T3, js, ss, ab + x, val, a.cand, a.cap, a.count);
                    }
                }
                continue;
            }
            // phase 3 over the whole piece
            exh += pend - px0;
            Word<L> v[D + 1];
            const uint64_t y0 = ybase + px0 + (uint64_t)lane;
#pragma unroll
            for (int jj = 0; jj <= D; jj++) v[jj] = poly_at<L, D>(c, y0 + 32ull * (uint64_t)jj);
#pragma unroll
            for (int lev = 1; lev <= D; lev++)
#pragma unroll
                for (int jj = D; jj >= lev; jj--) w_sub<L>(v[jj], v[jj - 1]);
            const uint32_t trips = (pend - px0 + 31u) >> 5;
#pragma unroll 1
            for (uint32_t t = 0; t < trips; t++) {
                const uint32_t x = px0 + t * 32u + (uint32_t)lane;
                const uint64_t val = v[0].l[L - 1] + jb.shift3;
                emit_warp(x < pend && val < jb.T3, js, ss, ab + x, val, a.cand, a.cap, a.count);
#pragma unroll
                for (int l = 0; l < D; l++) w_add<L>(v[l], v[l + 1]);
            }
        }
    }
    if (lane == 0 && exh) atomicAdd((unsigned long long*)&a.stats[ST_EXH], (unsigned long long)exh);
    if (lane == 0 && refined) atomicAdd((unsigned long long*)&a.stats[ST_REF], (unsigned long long)refined);
}

// Lines per packet held in shared memory between the two phases of a task.
constexpr int NU_MAX = 8;
constexpr int WARPS_PER_CTA = 8;
constexpr int TASK_LINES = 32 * NU_MAX;

// Line s of a task (packet s / nu, line s % nu of that packet) sits at
// stage_slot(s): one padding slot per 32 keeps both the packet-major writes
// of phase 1 (stride nu between lanes) and the line-major reads of phase 2
// (stride 1) free of shared-memory bank conflicts.
__device__ __forceinline__ int stage_slot(int s) { return s + (s >> 5); }

struct LineStage {
    uint64_t B[TASK_LINES + TASK_LINES / 32];
    uint64_t A[TASK_LINES + TASK_LINES / 32];
    uint32_t n[TASK_LINES + TASK_LINES / 32];   // arguments of the line; 0 = no line
    uint32_t blk[32];                            // block of each packet
    uint32_t i0[32];                             // first sub-interval of each packet in its block
};

// Phase 1: each lane steps the tabulated differences of its packet and parks
// the search words and lengths of its nu lines in shared memory.  Phase 2:
// the warp searches the task's lines 32 at a time in sub-interval order, so
// that the 32 lines searched together are neighbouring sub-intervals: their
// slopes differ in the low bits only, their continued fractions share all
// but the last partial quotients, and the lanes take the same branches of
// the search loop.  Only the search state is live in phase 2 (the W-bit
// packet state is dead by then); block fields are reloaded only on the rare
// resolve path.
// G = false: jobs with the regular filter and the literal threshold only
// (the hot path, no other code in the kernel); G = true: jobs that may use
// Lefevre's filter or the sound mode.
template <int L, int D, bool G>
__device__ __forceinline__ void fused_task(const DevTask& t, const LaunchArgs& a, LineStage& st,
                                           uint32_t& st_lines, uint32_t& st_fail, uint32_t& st_half,
                                           uint16_t* fl) {
    const int lane = threadIdx.x & 31;
    const uint32_t nu = a.jobs[t.job].nu;
    {
        // the job record stays in global memory (a local copy of the whole
        // record would be written to the stack at every task)
        const DevJob& job = a.jobs[t.job];
        Packet<L, D> P;
        const uint32_t bi = packet_init<L, D>(P, t, job, a);
        st.blk[lane] = bi;
        st.i0[lane] = P.i0;
        const uint32_t N = 1u << job.log2_N;
        const uint64_t shift = job.shift;
        // one line: its search words and length to the stage, one step
        auto park = [&](uint32_t it) {
            uint64_t B, A;
            packet_words<L, D>(P, shift, B, A);
            const uint32_t i = P.i0 + it;
            const bool valid = P.active && i < P.i1;
            const int s = stage_slot(lane * (int)nu + (int)it);
            st.B[s] = B;
            st.A[s] = A;
            st.n[s] = valid ? (uint32_t)min((uint64_t)N, P.blk.length - (uint64_t)i * N) : 0u;
            packet_step<L, D>(P);
        };
        if (a.unroll >= 2 && (nu & 1u) == 0) {
            // difference steps two at a time (a tiling knob)
#pragma unroll 1
            for (uint32_t it = 0; it < nu; it += 2) {
                park(it);
                park(it + 1);
            }
        } else {
#pragma unroll 1
            for (uint32_t it = 0; it < nu; it++) park(it);
        }
    }
    __syncwarp();
    const uint64_t Tm = a.jobs[t.job].Tm;
    const bool lefevre = G && (a.jobs[t.job].flags & TMD_LEFEVRE) != 0;
    // lanes per line in the filter (a tiling knob: 1, 2 or 4): line s of a
    // round is split into lp pieces of consecutive arguments, each lane
    // bounding its piece's own line (B - A x0, A) over fewer points; the
    // line fails when one of its pieces does, and its first lane carries it
    const uint32_t lpl = a.lanes >= 4 ? 2u : (a.lanes >= 2 ? 1u : 0u);
    const uint32_t lp = 1u << lpl, piece = (uint32_t)lane & (lp - 1u);
    uint32_t nfail = 0;  // general variant: failing lines listed in fl (warp-uniform)
    // one lane per line (the default) has a loop of its own: the pieces'
    // bookkeeping costs the hot loop registers and ~2.5 % when shared
    if (lpl == 0) {
#pragma unroll 1
    for (uint32_t r = 0; r < nu; r++) {
        const int s = (int)r * 32 + lane;
        const int slot = stage_slot(s);
        const uint32_t n = st.n[slot];
        const uint64_t B = st.B[slot];
        const uint64_t A = st.A[slot];
        uint32_t hs = 0;
        uint64_t lb = ~0ull;
        if (n) lb = lefevre ? lefevre_lower_bound<true>(B, A, n, &hs) : cf_lower_bound(B, A, n, &hs);
        const bool fail = n && lb < Tm;
        st_lines += n ? 1u : 0u;
        st_fail += fail ? 1u : 0u;
        st_half += hs;
        if (G) {
            // general variant: the failing lines of the task are listed and
            // resolved 32 at a time below (one lane each), not round by round
            // with a few active lanes
            const unsigned fm = __ballot_sync(FULLMASK, fail);
            if (fail) fl[nfail + (uint32_t)__popc(fm & ((1u << lane) - 1u))] = (uint16_t)s;
            nfail += (uint32_t)__popc(fm);
        } else if (__any_sync(FULLMASK, fail)) {
            const uint32_t pk = (uint32_t)s / nu;
            const uint32_t i = st.i0[pk] + (uint32_t)s % nu;
            const DevBlock& bk = a.blocks[st.blk[pk]];
            const DevJob& jb = a.jobs[t.job];
            resolve_and_emit(fail, B, A, n ? n : 1u, Tm, (jb.flags & TMD_ALL_HITS) != 0, t.job,
                             (uint32_t)(bk.first_sub + i), bk.start + ((uint64_t)i << jb.log2_N), a.cand,
                             a.cap, a.count);
        }
    }
    } else {
#pragma unroll 1
    for (uint32_t r = 0; r < (nu << lpl); r++) {
        const int s = (int)(((r << 5) + (uint32_t)lane) >> lpl);
        const int slot = stage_slot(s);
        const uint32_t n = st.n[slot];
        const uint64_t B = st.B[slot];
        const uint64_t A = st.A[slot];
        uint32_t np = n;
        uint64_t Bp = B;
        if (lpl) {
            const uint32_t w = (n + lp - 1u) >> lpl, x0 = piece * w;
            np = n > x0 ? min(w, n - x0) : 0u;
            Bp = B - A * (uint64_t)x0;
        }
        uint32_t hs = 0;
        uint64_t lb = ~0ull;
        if (np) lb = lefevre ? lefevre_lower_bound<true>(Bp, A, np, &hs) : cf_lower_bound(Bp, A, np, &hs);
        bool fail = np && lb < Tm;
        if (lpl) {
            unsigned f = fail ? 1u : 0u;
            for (uint32_t off = 1; off < lp; off <<= 1) f |= __shfl_xor_sync(FULLMASK, f, (int)off);
            fail = f != 0 && piece == 0;
        }
        st_lines += (n && piece == 0) ? 1u : 0u;
        st_fail += fail ? 1u : 0u;
        st_half += hs;
        if (G) {
            // general variant: the failing lines of the task are listed and
            // resolved 32 at a time below (one lane each), not round by round
            // with a few active lanes
            const unsigned fm = __ballot_sync(FULLMASK, fail);
            if (fail) fl[nfail + (uint32_t)__popc(fm & ((1u << lane) - 1u))] = (uint16_t)s;
            nfail += (uint32_t)__popc(fm);
        } else if (__any_sync(FULLMASK, fail)) {
            const uint32_t pk = (uint32_t)s / nu;
            const uint32_t i = st.i0[pk] + (uint32_t)s % nu;
            const DevBlock& bk = a.blocks[st.blk[pk]];
            const DevJob& jb = a.jobs[t.job];
            resolve_and_emit(fail, B, A, n ? n : 1u, Tm, (jb.flags & TMD_ALL_HITS) != 0, t.job,
                             (uint32_t)(bk.first_sub + i), bk.start + ((uint64_t)i << jb.log2_N), a.cand,
                             a.cap, a.count);
        }
    }
    }
    if (G && nfail) {
        __syncwarp();
        const DevJob& jb = a.jobs[t.job];
        const bool all_hits = (jb.flags & TMD_ALL_HITS) != 0;
#pragma unroll 1
        for (uint32_t base = 0; base < nfail; base += 32) {
            const uint32_t k = base + (uint32_t)lane;
            const bool act = k < nfail;
            const int s = act ? (int)fl[k] : 0;
            const int slot = stage_slot(s);
            const uint32_t n = act ? st.n[slot] : 1u;
            const uint64_t B = st.B[slot];
            const uint64_t A = st.A[slot];
            const uint32_t pk = (uint32_t)s / nu;
            const uint32_t i = st.i0[pk] + (uint32_t)s % nu;
            const DevBlock& bk = a.blocks[st.blk[pk]];
            if (jb.flags & TMD_SOUND)
                sound_exhaustive<L, D>(act, B, A, n, bk.table_off, i, (uint32_t)(bk.first_sub + i),
                                       bk.start + ((uint64_t)i << jb.log2_N), t.job, jb, a);
            else
                resolve_and_emit(act, B, A, n, Tm, all_hits, t.job, (uint32_t)(bk.first_sub + i),
                                 bk.start + ((uint64_t)i << jb.log2_N), a.cand, a.cap, a.count);
        }
    }
    __syncwarp();
}

template <int L, int D>
__device__ __forceinline__ void generate_task(const DevTask& t, const LaunchArgs& a) {
    const DevJob& job = a.jobs[t.job];
    Packet<L, D> P;
    packet_init<L, D>(P, t, job, a);
#pragma unroll 1
    for (uint32_t it = 0; it < job.nu; it++) {
        const uint32_t i = P.i0 + it;
        if (P.active && i < P.i1) {
            uint64_t B, A;
            packet_words<L, D>(P, job.shift, B, A);
            const uint64_t line = job.line_off + P.blk.first_sub + i;
            a.lin_B[line] = B;
            a.lin_A[line] = A;
        }
        packet_step<L, D>(P);
    }
}

// ------------------------------------------------------------------- kernels
// The plain form runs 4-warp CTAs (finer-grained scheduling of the last
// wave than 8-warp CTAs).
constexpr int FUSED_WARPS_PER_CTA = 4;

// Register caps (3 CTAs of 256 threads per SM, 6 of 128): the search needs
// ~75 registers; the rarely called non-inlined resolve and exhaustive paths
// would otherwise set the kernels' register counts and cut their occupancy,
// so they spill instead.
template <int L, int D, bool G>
__global__ void __launch_bounds__(128, 6) k_fused(LaunchArgs a) {
    __shared__ LineStage stage[FUSED_WARPS_PER_CTA];
    __shared__ uint16_t fails[G ? FUSED_WARPS_PER_CTA * TASK_LINES : 1];
    const uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= a.n_tasks) return;  // whole warp
    uint32_t sl = 0, sf = 0, sh = 0;
    const DevTask t = a.tasks[w];
    fused_task<L, D, G>(t, a, stage[threadIdx.x >> 5], sl, sf, sh, fails + (G ? (threadIdx.x >> 5) * TASK_LINES : 0));
    flush_stats(a.stats, sl, sf, sh);
}

template <int L, int D>
__global__ void __launch_bounds__(256) k_generate(LaunchArgs a) {
    const uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= a.n_tasks) return;
    const DevTask t = a.tasks[w];
    generate_task<L, D>(t, a);
}

// Persistent form: a grid of resident CTAs per (limbs, degree) class; each
// warp takes the next task of its class from a device counter until the
// class's list is exhausted (no waiting on other warps: one atomicAdd per
// task).
template <int L, int D, bool G>
__global__ void __launch_bounds__(256, 3) k_persistent(LaunchArgs a) {
    __shared__ LineStage stage[WARPS_PER_CTA];
    __shared__ uint16_t fails[G ? WARPS_PER_CTA * TASK_LINES : 1];
    LineStage& stg = stage[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    uint32_t sl = 0, sf = 0, sh = 0;
    for (;;) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(a.queue_head, 1u);
        t = __shfl_sync(FULLMASK, t, 0);
        if ((uint64_t)t >= a.n_tasks) break;
        const DevTask task = a.tasks[t];
        fused_task<L, D, G>(task, a, stg, sl, sf, sh, fails + (G ? (threadIdx.x >> 5) * TASK_LINES : 0));
    }
    flush_stats(a.stats, sl, sf, sh);
}

// Sound jobs in the line search: phases 2 and 3 (sound_exhaustive) for the
// lanes of one job at a time, so that the job record and its (limbs,
// degree) instantiation are uniform across the warp.
__device__ __noinline__ void sound_lines(bool fail, uint64_t B, uint64_t A, uint32_t n, uint64_t table_off,
                                         uint32_t i, uint32_t sub, uint64_t arg_base, uint32_t job,
                                         const DevJob& jb, const LaunchArgs& la) {
    switch (jb.L * 8 + jb.d) {
#define TMD_SOUND_CASE(L, D)                                                                     \
    case L * 8 + D:                                                                              \
        sound_exhaustive<L, D>(fail, B, A, n, table_off, i, sub, arg_base, job, jb, la);          \
        break;
        TMD_SOUND_CASE(1, 1) TMD_SOUND_CASE(1, 2) TMD_SOUND_CASE(1, 3) TMD_SOUND_CASE(1, 4)
        TMD_SOUND_CASE(2, 1) TMD_SOUND_CASE(2, 2) TMD_SOUND_CASE(2, 3) TMD_SOUND_CASE(2, 4)
        TMD_SOUND_CASE(3, 1) TMD_SOUND_CASE(3, 2) TMD_SOUND_CASE(3, 3) TMD_SOUND_CASE(3, 4)
#undef TMD_SOUND_CASE
        default:
            break;
    }
}

// Line search.  JOBS: the lines written by k_generate for the resident plan
// (line index -> job -> block by binary search; sound jobs continue with
// phases 2 and 3 from the block tables).  RAW: caller arrays with per-line
// lengths; record = (0, line, x, value).

template <bool RAW>
__global__ void __launch_bounds__(256) k_search_lines(LineArgs a) {
    const uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t s = (w << 5) + (threadIdx.x & 31);
    if ((w << 5) >= a.n_lines) return;  // whole warp
    const bool valid = s < a.n_lines;
    uint64_t B = 0, A = 0, Tm = a.Tm, arg_base = 0, table_off = 0;
    uint32_t n = 1, job = 0, sub = 0, flags = a.flags, iblk = 0;
    if (valid) {
        B = a.B[s];
        A = a.A[s];
        if (RAW) {
            uint32_t ln = a.len[s];
            if (ln == 0 || ln > 65536u) {
                atomicOr(a.err, 1u);
                ln = ln == 0 ? 1u : 65536u;
            }
            n = ln;
            sub = (uint32_t)s;
        } else {
            uint32_t lo = 0, hi = a.n_jobs - 1;
            while (lo < hi) {
                uint32_t mid = (lo + hi + 1) >> 1;
                if (a.jobs[mid].line_off <= s) lo = mid; else hi = mid - 1;
            }
            const DevJob& jb = a.jobs[lo];
            job = lo;
            Tm = jb.Tm;
            flags = jb.flags;
            const uint64_t js = s - jb.line_off;
            uint32_t b0 = jb.block_off, b1 = jb.block_off + jb.n_blocks - 1;
            while (b0 < b1) {
                uint32_t mid = (b0 + b1 + 1) >> 1;
                if (a.blocks[mid].first_sub <= js) b0 = mid; else b1 = mid - 1;
            }
            const DevBlock& bk = a.blocks[b0];
            const uint64_t i = js - bk.first_sub;
            const uint64_t N = 1ull << jb.log2_N;
            n = (uint32_t)min(N, bk.length - i * N);
            sub = (uint32_t)js;
            arg_base = bk.start + i * N;
            table_off = bk.table_off;
            iblk = (uint32_t)i;
        }
    }
    uint32_t hs = 0;
    uint64_t lb = ~0ull;
    if (valid) lb = (flags & TMD_LEFEVRE) ? lefevre_lower_bound<true>(B, A, n, &hs) : cf_lower_bound(B, A, n, &hs);
    const bool fail = valid && lb < Tm;
    const bool sound = !RAW && valid && (flags & TMD_SOUND);
    // all lanes of a warp share ALL_HITS in practice; take the warp's OR
    const bool all_hits = __any_sync(FULLMASK, valid && (flags & TMD_ALL_HITS));
    if (__any_sync(FULLMASK, fail && !sound))
        resolve_and_emit(fail && !sound, B, A, n, Tm, all_hits, job, sub, arg_base, a.cand, a.cap, a.count);
    if (!RAW) {
        unsigned todo = __ballot_sync(FULLMASK, sound && fail);
        if (todo) {
            LaunchArgs la;
            la.jobs = a.jobs;
            la.blocks = a.blocks;
            la.tables = a.tables;
            la.tasks = nullptr;
            la.n_tasks = 0;
            la.lin_B = la.lin_A = nullptr;
            la.cand = a.cand;
            la.cap = a.cap;
            la.count = a.count;
            la.stats = a.stats;
            la.queue_head = nullptr;
            la.lanes = la.unroll = 0;
            while (todo) {
                const uint32_t jl = __shfl_sync(FULLMASK, job, __ffs(todo) - 1);
                const bool mine = sound && fail && job == jl;
                todo &= ~__ballot_sync(FULLMASK, mine);
                sound_lines(mine, B, A, n, table_off, iblk, sub, arg_base, jl, a.jobs[jl], la);
            }
        }
    }
    flush_stats(a.stats, valid ? 1u : 0u, fail ? 1u : 0u, hs);
}

// MODE 0: Algorithm 4; 1: Algorithm 3; 2: Algorithm 3 with the specific instructions
template <int MODE>
__global__ void __launch_bounds__(256) k_lower_bounds(const uint64_t* B, const uint64_t* A,
                                                      const uint32_t* len, uint64_t n, uint64_t* lb,
                                                      uint32_t* hs_out, uint32_t* err) {
    const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    uint32_t ln = len[s];
    if (ln == 0 || ln > 65536u) {
        atomicOr(err, 1u);
        ln = ln == 0 ? 1u : 65536u;
    }
    uint32_t hs = 0;
    lb[s] = MODE == 0 ? cf_lower_bound(B[s], A[s], ln, &hs)
                      : (MODE == 1 ? lefevre_lower_bound<false>(B[s], A[s], ln, &hs)
                                   : lefevre_lower_bound<true>(B[s], A[s], ln, &hs));
    if (hs_out) hs_out[s] = hs;
}

// ------------------------------------------------------- device planning
// Block and task records from the per-job segment table (Sect. III-A split
// and Sect. IV blocks: blocks of T arguments from each segment start, the
// last one of a segment shorter; packets of nu sub-intervals per block).
// One thread per block record and per task record (one launch for both);
// thread 0 also clears the plan's error word before the table kernels run,
// and, when given, the first threads clear a search's counters (n_misc
// statistics and error words and the candidate count).
// Blocks: the last job whose first block is <= b.  Tasks are laid out class
// by class (class_jobs lists the jobs of each (limbs, degree) class in
// order; class_task0 their first task), 32 packets per task within a job.
__device__ __forceinline__ void plan_records(uint64_t i, const DevJob* jobs, uint32_t n_jobs, DevBlock* blocks,
                                             uint64_t n_blocks, const uint32_t* class_jobs,
                                             const uint64_t* class_task0, uint32_t n_entries, DevTask* tasks,
                                             uint64_t n_tasks, uint32_t* plan_err, uint64_t* misc, uint32_t n_misc,
                                             uint64_t* count) {
    if (i == 0) *plan_err = 0;
    if (misc && i < n_misc) misc[i] = 0;
    if (count && i == 0) *count = 0;
    if (i < n_blocks) {
        uint32_t lo = 0, hi = n_jobs - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (jobs[mid].block_off <= i) lo = mid; else hi = mid - 1;
        }
        blocks[i] = block_record(jobs[lo], lo, i - jobs[lo].block_off);
    }
    if (i < n_tasks) {
        uint32_t lo = 0, hi = n_entries - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (class_task0[mid] <= i) lo = mid; else hi = mid - 1;
        }
        const uint32_t j = class_jobs[lo];
        tasks[i] = task_record(jobs[j], j, i - class_task0[lo]);
    }
}

__global__ void __launch_bounds__(256) k_plan(const DevJob* jobs, uint32_t n_jobs, DevBlock* blocks, uint64_t n_blocks,
                                              const uint32_t* class_jobs, const uint64_t* class_task0,
                                              uint32_t n_entries, DevTask* tasks, uint64_t n_tasks,
                                              uint32_t* plan_err, uint64_t* misc, uint32_t n_misc,
                                              uint64_t* count) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    plan_records(i, jobs, n_jobs, blocks, n_blocks, class_jobs, class_task0, n_entries, tasks, n_tasks, plan_err,
                 misc, n_misc, count);
}

// The same with the uploaded part of a small plan (job records and class
// lists, n_words words) passed as the kernel's parameter instead of copied
// to the device first: the threads read the records from the parameter and
// write them to the arena's start for the kernels that follow.
__global__ void __launch_bounds__(256) k_plan_inline(const __grid_constant__ InlinePlan src, uint32_t n_words,
                                                     uint64_t* arena, uint32_t n_jobs, uint64_t o_cjobs,
                                                     uint64_t o_ctask, uint32_t n_entries, uint64_t o_blocks,
                                                     uint64_t n_blocks, uint64_t o_tasks, uint64_t n_tasks,
                                                     uint32_t* plan_err, uint64_t* misc, uint32_t n_misc,
                                                     uint64_t* count) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_words) arena[i] = src.w[i];
    const char* base = (const char*)src.w;
    char* a = (char*)arena;
    plan_records(i, (const DevJob*)base, n_jobs, (DevBlock*)(a + o_blocks), n_blocks,
                 (const uint32_t*)(base + o_cjobs), (const uint64_t*)(base + o_ctask), n_entries,
                 (DevTask*)(a + o_tasks), n_tasks, plan_err, misc, n_misc, count);
}

cudaError_t launch_plan(const DevJob* jobs, uint32_t n_jobs, DevBlock* blocks, uint64_t n_blocks,
                        const uint32_t* class_jobs, const uint64_t* class_task0, uint32_t n_entries,
                        DevTask* tasks, uint64_t n_tasks, uint32_t* plan_err, uint64_t* misc, uint32_t n_misc,
                        uint64_t* count, cudaStream_t s) {
    const uint64_t n = n_blocks > n_tasks ? n_blocks : n_tasks;
    k_plan<<<(unsigned)((n + 255) / 256 + (n == 0)), 256, 0, s>>>(jobs, n_jobs, blocks, n_blocks, class_jobs,
                                                                   class_task0, n_entries, tasks, n_tasks, plan_err,
                                                                   misc, n_misc, count);
    return cudaGetLastError();
}

cudaError_t launch_plan_inline(const InlinePlan& src, uint32_t n_words, uint64_t* arena, uint32_t n_jobs,
                               uint64_t o_cjobs, uint64_t o_ctask, uint32_t n_entries, uint64_t o_blocks,
                               uint64_t n_blocks, uint64_t o_tasks, uint64_t n_tasks, uint32_t* plan_err,
                               uint64_t* misc, uint32_t n_misc, uint64_t* count, cudaStream_t s) {
    uint64_t n = n_blocks > n_tasks ? n_blocks : n_tasks;
    if (n < n_words) n = n_words;
    k_plan_inline<<<(unsigned)((n + 255) / 256 + (n == 0)), 256, 0, s>>>(
        src, n_words, arena, n_jobs, o_cjobs, o_ctask, n_entries, o_blocks, n_blocks, o_tasks, n_tasks, plan_err,
        misc, n_misc, count);
    return cudaGetLastError();
}

// The statistics and error words (n_misc words) and a candidate count, in one
// launch instead of two memsets.
__global__ void k_zero_counters(uint64_t* misc, uint32_t n_misc, uint64_t* count) {
    const uint32_t i = threadIdx.x;
    if (i < n_misc) misc[i] = 0;
    if (i == 0 && count) *count = 0;
}

// The candidate count and three error words of a search into mapped host
// memory (one launch and one wait instead of two copies).
__global__ void k_readback(const uint64_t* count, const uint32_t* words, uint64_t* host) {
    if (threadIdx.x == 0) {
        host[0] = *count;
        host[1] = (uint64_t)words[0] | ((uint64_t)words[1] << 32);
        host[2] = words[2];
    }
}

cudaError_t launch_readback(const uint64_t* count, const uint32_t* words, uint64_t* host, cudaStream_t s) {
    k_readback<<<1, 32, 0, s>>>(count, words, host);
    return cudaGetLastError();
}

cudaError_t launch_zero_counters(uint64_t* misc, uint32_t n_misc, uint64_t* count, cudaStream_t s) {
    k_zero_counters<<<1, 32, 0, s>>>(misc, n_misc, count);
    return cudaGetLastError();
}

// ---------------------------------------------------------- block tables
// One thread per Taylor block: correctly rounded coefficients of R_t and the
// 2d+1 step-N difference words (the host path runs the same routine).  Pass
// 0 works with 384-bit words and 32 guard bits; pass 1, a kernel of its own
// (its wider code stays out of pass 0's instruction cache), redoes only the
// blocks left undecided, at 512 bits with 64 guard bits, then at 768 bits
// with 320 (Ziv); a block still undecided raises ERR_ROUNDING in the error
// word.  (The per-job anchors of
// the host path are not used here: on the device the anchor's own
// evaluation would sit in front of every block's on the critical path.)
__constant__ CoeffConsts c_coeff;

__device__ __forceinline__ CoeffJob block_coeff_job(const DevJob& jb, int e_out) {
    CoeffJob J;
    J.func = jb.func;
    J.e_in = jb.e_in;
    J.p = jb.p;
    J.d = (int)jb.d;
    J.L = (int)jb.L;
    J.scale_log2 = (jb.flags & TMD_BP_DIRECTED) ? jb.p - e_out : jb.p + 1 - e_out;
    J.log2_N = (int)jb.log2_N;
    J.red = reduction_exponent(jb.func, jb.e_in, e_out);
    return J;
}

// One instantiation per function F (exp, 2^x, log): each holds only its own
// enclosure and coefficient code, so a warp fetches less code (the kernel
// waits on instruction fetches: the served 10k-job stream ran 1.4-1.6e14
// args/s with one kernel for all three functions, 1.7-1.9e14 with three);
// the blocks of the other functions return at once.  LPB threads per block:
// with few blocks (one wave of a few warps per SM) the kernel is bound by the
// latency of each thread's serial multiword chain, so LPB = 4 consecutive
// lanes share a block -- each forms f(X_t), rounds the orders k with k % 4
// equal to its part and writes a quarter of the words, the coefficients
// passing through shared memory -- and a block's table is kept only if all
// four parts' roundings were decided.
// threads per CTA: 64 with four threads per block (small plans: one wave of
// a few warps per SM, more SMs fetching the code in parallel), 256 with one
// (large plans: several warps per scheduler share the fetched code; the
// served groups' tables ran 0.85-0.97x the time of 64-thread CTAs)
template <int LPB>
__host__ __device__ constexpr int table_tpb() {
    return LPB > 1 ? 64 : 256;
}

template <int F, int LPB>
__global__ void __launch_bounds__(table_tpb<LPB>()) k_block_tables(const DevJob* jobs, const DevBlock* blocks,
                                                            uint64_t n_blocks, uint64_t* tables, uint32_t* status,
                                                            const uint64_t* ctab) {
    static_assert(LPB == 1 || LPB == 2 || LPB == 4, "a block's parts are consecutive lanes of one warp");
    constexpr int NC = (COEFF_MAX_DEG + 1) * COEFF_MAX_LIMBS;
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (LPB == 1) {
        const uint64_t b = g;
        if (b >= n_blocks) return;
        const DevBlock bk = blocks[b];
        const DevJob jb = jobs[bk.job];
        if (jb.func != F) return;
        CoeffJob J = block_coeff_job(jb, bk.e_out);
        J.func = F;
        const uint64_t M = (1ull << (jb.p - 1)) + bk.start;
        uint64_t c[NC];
        // 384 bits with 32 guard bits below the coefficients' last place: an
        // undecided rounding (odds ~2^-40 per coefficient) or a job whose
        // words need more bits goes to k_block_tables_wide (512, then 768 bits)
        const bool ok = block_coeffs<6>(J, M, 32, c_coeff, c, nullptr, ctab);
        if (ok) block_table_words(J, c, tables + bk.table_off);
        if (ok && (jb.flags & TMD_SOUND)) coeffs_packed(J, c, tables + bk.table_off + (2 * J.d + 1) * J.L);
        status[b] = ok ? 0 : 1;
        return;
    }
    __shared__ uint64_t sc[LPB > 1 ? table_tpb<LPB>() / LPB : 1][NC];
    const uint64_t b = g / LPB;
    const int part = (int)(g % LPB);
    bool act = b < n_blocks;
    DevBlock bk;
    DevJob jb;
    CoeffJob J;
    if (act) {
        bk = blocks[b];
        jb = jobs[bk.job];
        act = jb.func == F;
    }
    bool ok = false;
    uint64_t* c = sc[threadIdx.x / LPB];
    if (act) {
        J = block_coeff_job(jb, bk.e_out);
        J.func = F;
        const uint64_t M = (1ull << (jb.p - 1)) + bk.start;
        ok = block_coeffs<6>(J, M, 32, c_coeff, c, nullptr, ctab, part, LPB);
    }
    // every lane of the warp votes (inactive ones with ok = false): the vote
    // must not sit behind a short-circuited condition
    const unsigned vote = __ballot_sync(0xffffffffu, ok);
    const unsigned lane = threadIdx.x & 31u;
    const unsigned mine = ((1u << LPB) - 1u) << (lane & ~(unsigned)(LPB - 1));
    const bool all_ok = act && (vote & mine) == mine;
    __syncwarp();
    if (all_ok) block_table_words(J, c, tables + bk.table_off, part, LPB);
    if (all_ok && part == 0 && (jb.flags & TMD_SOUND))
        coeffs_packed(J, c, tables + bk.table_off + (2 * J.d + 1) * J.L);
    if (act && part == 0) status[b] = all_ok ? 0 : 1;
}

__global__ void __launch_bounds__(64) k_block_tables_wide(const DevJob* jobs, const DevBlock* blocks,
                                                          uint64_t n_blocks, uint64_t* tables, uint32_t* status,
                                                          uint32_t* err, const uint64_t* ctab) {
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_blocks || status[b] == 0) return;
    const DevBlock bk = blocks[b];
    const DevJob jb = jobs[bk.job];
    const CoeffJob J = block_coeff_job(jb, bk.e_out);
    const uint64_t M = (1ull << (jb.p - 1)) + bk.start;
    uint64_t c[(COEFF_MAX_DEG + 1) * COEFF_MAX_LIMBS];
    if (block_coeffs<8>(J, M, 64, c_coeff, c, nullptr, ctab) ||
        block_coeffs<12>(J, M, 320, c_coeff, c, nullptr, ctab)) {
        block_table_words(J, c, tables + bk.table_off);
        if (jb.flags & TMD_SOUND) coeffs_packed(J, c, tables + bk.table_off + (2 * J.d + 1) * J.L);
        status[b] = 0;
    } else {
        atomicOr(err, (uint32_t)ERR_ROUNDING);
    }
}

cudaError_t upload_coeff_consts(const CoeffConsts& C) {
    return cudaMemcpyToSymbol(c_coeff, &C, sizeof C);
}

// The exp and 2^x tables of the table-driven enclosures (coeffs.cuh), one
// thread per entry; an entry that fails to enclose sets *err.
__global__ void __launch_bounds__(64) k_coeff_tables(uint64_t* ctab, uint32_t* err) {
    const int e = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= CT_BASES * CT_LEVELS * CT_ENTRIES) return;
    const int base = e / (CT_LEVELS * CT_ENTRIES), level = (e / CT_ENTRIES) % CT_LEVELS, b = e % CT_ENTRIES;
    if (!ct_entry(base, level, b, c_coeff, ctab + ct_index(base, level, b, 0), ctab + ct_index(base, level, b, 1)))
        atomicOr(err, 1u);
}

cudaError_t launch_coeff_tables(uint64_t* ctab, uint32_t* err, cudaStream_t s) {
    const int n = CT_BASES * CT_LEVELS * CT_ENTRIES;
    k_coeff_tables<<<(n + 63) / 64, 64, 0, s>>>(ctab, err);
    return cudaGetLastError();
}

// func_mask: bit f set when the plan holds blocks of function f
// plans of up to this many blocks take four threads per block (16 k blocks:
// 64 k threads, ~13 warps per SM)
constexpr uint64_t TABLE_SPLIT_MAX_BLOCKS = 16384;

cudaError_t launch_block_tables(const DevJob* jobs, const DevBlock* blocks, uint64_t n_blocks, uint64_t* tables,
                                uint32_t* status, uint32_t* err, const uint64_t* ctab, uint32_t func_mask,
                                cudaStream_t s) {
    if (n_blocks == 0) return cudaSuccess;
    // 64-thread CTAs spread the (few, long) threads over more SMs; four
    // threads per block while the plan is one wave of a few warps per SM
    const unsigned grid = (unsigned)((n_blocks + 63) / 64);
    if (n_blocks <= TABLE_SPLIT_MAX_BLOCKS) {
        constexpr int T4 = table_tpb<4>();
        const unsigned g4 = (unsigned)((4 * n_blocks + T4 - 1) / T4);
        if (func_mask & 1u) k_block_tables<0, 4><<<g4, T4, 0, s>>>(jobs, blocks, n_blocks, tables, status, ctab);
        if (func_mask & 2u) k_block_tables<1, 4><<<g4, T4, 0, s>>>(jobs, blocks, n_blocks, tables, status, ctab);
        if (func_mask & 4u) k_block_tables<2, 4><<<g4, T4, 0, s>>>(jobs, blocks, n_blocks, tables, status, ctab);
    } else {
        constexpr int T1 = table_tpb<1>();
        const unsigned g1 = (unsigned)((n_blocks + T1 - 1) / T1);
        if (func_mask & 1u) k_block_tables<0, 1><<<g1, T1, 0, s>>>(jobs, blocks, n_blocks, tables, status, ctab);
        if (func_mask & 2u) k_block_tables<1, 1><<<g1, T1, 0, s>>>(jobs, blocks, n_blocks, tables, status, ctab);
        if (func_mask & 4u) k_block_tables<2, 1><<<g1, T1, 0, s>>>(jobs, blocks, n_blocks, tables, status, ctab);
    }
    k_block_tables_wide<<<grid, 64, 0, s>>>(jobs, blocks, n_blocks, tables, status, err, ctab);
    return cudaGetLastError();
}

// --------------------------------------------------------------- launchers
typedef void (*TaskKernel)(LaunchArgs);

static TaskKernel fused_kernel(uint32_t L, uint32_t D, bool G) {
    static const TaskKernel tab[2][3][4] = {
        {{k_fused<1, 1, false>, k_fused<1, 2, false>, k_fused<1, 3, false>, k_fused<1, 4, false>},
         {k_fused<2, 1, false>, k_fused<2, 2, false>, k_fused<2, 3, false>, k_fused<2, 4, false>},
         {k_fused<3, 1, false>, k_fused<3, 2, false>, k_fused<3, 3, false>, k_fused<3, 4, false>}},
        {{k_fused<1, 1, true>, k_fused<1, 2, true>, k_fused<1, 3, true>, k_fused<1, 4, true>},
         {k_fused<2, 1, true>, k_fused<2, 2, true>, k_fused<2, 3, true>, k_fused<2, 4, true>},
         {k_fused<3, 1, true>, k_fused<3, 2, true>, k_fused<3, 3, true>, k_fused<3, 4, true>}}};
    return tab[G ? 1 : 0][L - 1][D - 1];
}

static TaskKernel generate_kernel(uint32_t L, uint32_t D) {
    static const TaskKernel tab[3][4] = {
        {k_generate<1, 1>, k_generate<1, 2>, k_generate<1, 3>, k_generate<1, 4>},
        {k_generate<2, 1>, k_generate<2, 2>, k_generate<2, 3>, k_generate<2, 4>},
        {k_generate<3, 1>, k_generate<3, 2>, k_generate<3, 3>, k_generate<3, 4>}};
    return tab[L - 1][D - 1];
}

cudaError_t launch_tasks(bool fused, uint32_t L, uint32_t D, bool G, const LaunchArgs& a, cudaStream_t s) {
    if (a.n_tasks == 0) return cudaSuccess;
    const uint64_t warps_per_cta = fused ? FUSED_WARPS_PER_CTA : 8;
    const uint64_t ctas = (a.n_tasks + warps_per_cta - 1) / warps_per_cta;
    TaskKernel k = fused ? fused_kernel(L, D, G) : generate_kernel(L, D);
    k<<<(unsigned)ctas, (unsigned)(32 * warps_per_cta), 0, s>>>(a);
    return cudaGetLastError();
}

static TaskKernel persistent_kernel(uint32_t L, uint32_t D, bool G) {
    static const TaskKernel tab[2][3][4] = {
        {{k_persistent<1, 1, false>, k_persistent<1, 2, false>, k_persistent<1, 3, false>, k_persistent<1, 4, false>},
         {k_persistent<2, 1, false>, k_persistent<2, 2, false>, k_persistent<2, 3, false>, k_persistent<2, 4, false>},
         {k_persistent<3, 1, false>, k_persistent<3, 2, false>, k_persistent<3, 3, false>, k_persistent<3, 4, false>}},
        {{k_persistent<1, 1, true>, k_persistent<1, 2, true>, k_persistent<1, 3, true>, k_persistent<1, 4, true>},
         {k_persistent<2, 1, true>, k_persistent<2, 2, true>, k_persistent<2, 3, true>, k_persistent<2, 4, true>},
         {k_persistent<3, 1, true>, k_persistent<3, 2, true>, k_persistent<3, 3, true>, k_persistent<3, 4, true>}}};
    return tab[G ? 1 : 0][L - 1][D - 1];
}

cudaError_t launch_persistent(uint32_t L, uint32_t D, bool G, const LaunchArgs& a, int ctas, cudaStream_t s) {
    persistent_kernel(L, D, G)<<<ctas, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t persistent_occupancy(uint32_t L, uint32_t D, bool G, int* blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, persistent_kernel(L, D, G), 256, 0);
}

cudaError_t launch_search_lines(bool raw, const LineArgs& a, cudaStream_t s) {
    if (a.n_lines == 0) return cudaSuccess;
    const uint64_t warps = (a.n_lines + 31) / 32;
    const uint64_t ctas = (warps + 7) / 8;
    if (raw)
        k_search_lines<true><<<(unsigned)ctas, 256, 0, s>>>(a);
    else
        k_search_lines<false><<<(unsigned)ctas, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_lower_bounds(int mode, const uint64_t* B, const uint64_t* A, const uint32_t* len,
                                uint64_t n, uint64_t* lb, uint32_t* hs, uint32_t* err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (mode == 2)
        k_lower_bounds<2><<<grid, 256, 0, s>>>(B, A, len, n, lb, hs, err);
    else if (mode == 1)
        k_lower_bounds<1><<<grid, 256, 0, s>>>(B, A, len, n, lb, hs, err);
    else
        k_lower_bounds<0><<<grid, 256, 0, s>>>(B, A, len, n, lb, hs, err);
    return cudaGetLastError();
}

}  // namespace tmd
