/* Brute-force minimum of (B - A x) mod 2^64 over 0 <= x < n, one line per
 * entry (Eq. (1) of Sect. II-A on 64-bit search words).
 *
 * TEST INFRASTRUCTURE ONLY (part of the CPU oracle): a plain loop over every
 * argument, used by the tests and by the timed CPU baseline; nothing on the
 * product path links or calls it.
 *
 * Unsigned 64-bit arithmetic in C is arithmetic mod 2^64, so B - A*x is the
 * value mod 2^64 directly.  The smallest x attaining the minimum is kept.
 * OpenMP splits the lines over threads (each line is independent).
 */
#include <stddef.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

void oracle_brute_min(size_t count, const uint64_t *B, const uint64_t *A,
                      const uint32_t *len, uint64_t *min_out, uint32_t *arg_out,
                      int threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (long long i = 0; i < (long long)count; i++) {
        uint64_t b = B[i], a = A[i];
        uint64_t best = UINT64_MAX;
        uint32_t arg = 0;
        uint32_t n = len[i];
        for (uint32_t x = 0; x < n; x++) {
            uint64_t v = b - a * (uint64_t)x;
            if (v < best) { best = v; arg = x; }
        }
        min_out[i] = best;
        arg_out[i] = arg;
    }
}

/* Every x with (B - A x) mod 2^64 < T, for every line: writes up to cap
 * (line, x, value) triples and returns the total number found. */
size_t oracle_brute_hits(size_t count, const uint64_t *B, const uint64_t *A,
                         const uint32_t *len, uint64_t T, uint32_t *line_out,
                         uint32_t *x_out, uint64_t *v_out, size_t cap)
{
    size_t found = 0;
    for (size_t i = 0; i < count; i++) {
        uint64_t b = B[i], a = A[i];
        for (uint32_t x = 0; x < len[i]; x++) {
            uint64_t v = b - a * (uint64_t)x;
            if (v < T) {
                if (found < cap) { line_out[found] = (uint32_t)i; x_out[found] = x; v_out[found] = v; }
                found++;
            }
        }
    }
    return found;
}

int oracle_threads_available(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
