/* Order-2 Markov text sampler for the synthetic inputs (host only).
 * cdf: (96*96) x 96 cumulative next-symbol distributions, row = 96*a + b for the
 * context (a, b) of the two previous symbols; alphabet: the 96 output bytes;
 * u: one uniform draw in [0,1) per output byte.  Initial context (0, 0). */
#include <stdint.h>

void markov_sample(const double* cdf, const uint8_t* alphabet, const double* u,
                   int64_t n, uint8_t* out) {
    const int K = 96;
    int a = 0, b = 0;
    for (int64_t t = 0; t < n; ++t) {
        const double* row = cdf + ((int64_t)a * K + b) * K;
        int lo = 0, hi = K - 1;           /* first index with row[i] > u[t] */
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (row[mid] > u[t]) hi = mid; else lo = mid + 1;
        }
        out[t] = alphabet[lo];
        a = b;
        b = lo;
    }
}
