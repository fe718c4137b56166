// Counter-based SplitMix64 (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014): value i of stream `seed` is
// the SplitMix64 finaliser applied to seed + (i+1) * 0x9E3779B97F4A7C15.
//
// The Gaussian projection of Sec. 3.2 / Eq. 3 (entries i.i.d. N(0,1), the
// 2-stable law) uses the Box-Muller transform on consecutive value pairs:
// u1 = (v_{2p} >> 11 + 1) 2^-53 in (0,1], u2 = (v_{2p+1} >> 11) 2^-53 in [0,1),
// entries 2p and 2p+1 (row-major [m][d]) are sqrt(-2 ln u1) cos(2 pi u2) and
// sqrt(-2 ln u1) sin(2 pi u2), computed in FP64 and rounded to FP32.
#include <cmath>

#include "pmlsh_impl.h"

uint64_t pm_splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void pm_gaussian_projection(uint64_t seed, int m, int d, float *A)
{
    const double two_pi = 6.283185307179586476925286766559;
    const int64_t total = (int64_t)m * d;
    for (int64_t p = 0; 2 * p < total; p++) {
        double u1 = ((double)(pm_splitmix64(seed, 2 * p) >> 11) + 1.0) * 0x1.0p-53;
        double u2 = (double)(pm_splitmix64(seed, 2 * p + 1) >> 11) * 0x1.0p-53;
        double rad = std::sqrt(-2.0 * std::log(u1));
        A[2 * p] = (float)(rad * std::cos(two_pi * u2));
        if (2 * p + 1 < total) A[2 * p + 1] = (float)(rad * std::sin(two_pi * u2));
    }
}
