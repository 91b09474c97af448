// Unsigned big integers for the host-side coefficient computation.
//
// Little-endian 64-bit limbs, kept trimmed (no zero top limb).  Only what the
// rigorous fixed-point evaluation of exp, 2^x and log needs: add, subtract,
// multiply, multiply/divide by a 64-bit word, shifts, comparison.
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

namespace tmd {

typedef unsigned __int128 u128;

struct Big {
    std::vector<uint64_t> v;

    Big() {}
    explicit Big(uint64_t x) { if (x) v.push_back(x); }

    static Big pow2(unsigned e) {
        Big r;
        r.v.assign(e / 64 + 1, 0);
        r.v[e / 64] = 1ull << (e % 64);
        return r;
    }
    bool zero() const { return v.empty(); }
    void trim() { while (!v.empty() && v.back() == 0) v.pop_back(); }
    uint64_t limb(size_t i) const { return i < v.size() ? v[i] : 0; }
    unsigned bits() const {
        if (v.empty()) return 0;
        return (unsigned)(64 * (v.size() - 1)) + 64 - (unsigned)__builtin_clzll(v.back());
    }
    bool bit(unsigned i) const { return (limb(i / 64) >> (i % 64)) & 1; }

    int cmp(const Big& o) const {
        if (v.size() != o.v.size()) return v.size() < o.v.size() ? -1 : 1;
        for (size_t i = v.size(); i-- > 0;)
            if (v[i] != o.v[i]) return v[i] < o.v[i] ? -1 : 1;
        return 0;
    }
    Big& add(const Big& o) {
        if (o.v.size() > v.size()) v.resize(o.v.size(), 0);
        uint64_t c = 0;
        for (size_t i = 0; i < v.size(); i++) {
            u128 s = (u128)v[i] + o.limb(i) + c;
            v[i] = (uint64_t)s;
            c = (uint64_t)(s >> 64);
        }
        if (c) v.push_back(c);
        return *this;
    }
    Big& add_u64(uint64_t a) { return add(Big(a)); }
    // requires *this >= o
    Big& sub(const Big& o) {
        uint64_t br = 0;
        for (size_t i = 0; i < v.size(); i++) {
            u128 d = (u128)v[i] - o.limb(i) - br;
            v[i] = (uint64_t)d;
            br = (uint64_t)(d >> 64) ? 1 : 0;
        }
        trim();
        return *this;
    }
    Big& mul_u64(uint64_t m) {
        if (m == 0) { v.clear(); return *this; }
        uint64_t c = 0;
        for (size_t i = 0; i < v.size(); i++) {
            u128 p = (u128)v[i] * m + c;
            v[i] = (uint64_t)p;
            c = (uint64_t)(p >> 64);
        }
        if (c) v.push_back(c);
        return *this;
    }
    // floor division by d (> 0); returns the remainder
    uint64_t div_u64(uint64_t d) {
        u128 r = 0;
        for (size_t i = v.size(); i-- > 0;) {
            u128 cur = (r << 64) | v[i];
            v[i] = (uint64_t)(cur / d);
            r = cur % d;
        }
        trim();
        return (uint64_t)r;
    }
    Big& shl(unsigned s) {
        if (v.empty() || s == 0) return *this;
        unsigned w = s / 64, b = s % 64;
        std::vector<uint64_t> r(v.size() + w + 1, 0);
        for (size_t i = 0; i < v.size(); i++) {
            r[i + w] |= v[i] << b;
            if (b) r[i + w + 1] |= v[i] >> (64 - b);
        }
        v.swap(r);
        trim();
        return *this;
    }
    Big& shr(unsigned s) {
        unsigned w = s / 64, b = s % 64;
        if (w >= v.size()) { v.clear(); return *this; }
        std::vector<uint64_t> r(v.size() - w, 0);
        for (size_t i = 0; i < r.size(); i++) {
            r[i] = v[i + w] >> b;
            if (b && i + w + 1 < v.size()) r[i] |= v[i + w + 1] << (64 - b);
        }
        v.swap(r);
        trim();
        return *this;
    }
    // true iff any of the low s bits is set
    bool low_bits_nonzero(unsigned s) const {
        for (unsigned i = 0; i < s / 64 && i < v.size(); i++)
            if (v[i]) return true;
        if (s % 64 && s / 64 < v.size()) return (v[s / 64] & ((1ull << (s % 64)) - 1)) != 0;
        return false;
    }
    static Big mul(const Big& a, const Big& b) {
        Big r;
        if (a.zero() || b.zero()) return r;
        r.v.assign(a.v.size() + b.v.size(), 0);
        for (size_t i = 0; i < a.v.size(); i++) {
            uint64_t c = 0;
            for (size_t j = 0; j < b.v.size(); j++) {
                u128 p = (u128)a.v[i] * b.v[j] + r.v[i + j] + c;
                r.v[i + j] = (uint64_t)p;
                c = (uint64_t)(p >> 64);
            }
            r.v[i + b.v.size()] = c;
        }
        r.trim();
        return r;
    }
};

inline Big shr_ceil(Big x, unsigned s) {  // ceil(x / 2^s)
    bool up = x.low_bits_nonzero(s);
    x.shr(s);
    if (up) x.add_u64(1);
    return x;
}

}  // namespace tmd
