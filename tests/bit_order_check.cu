// Host check of the bit-pattern order helpers of dfgks_device.cuh (nn_max, nn_min, nn_less,
// in_range, positive_bits) against fmax, fmin, < and >: bit for bit on non-negative values (zero,
// subnormals, normals, the overflow guards' bounds, infinity), and in_range and positive_bits on
// values of any sign, -0 and NaN included.
// Prints the number of mismatches; exit status 1 if there is any.
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <cmath>
#include <cfloat>
#include <vector>
#include "dfgks_device.cuh"

using namespace dfk;

static uint64_t state = 0x9E3779B97F4A7C15ull;
static uint64_t next_u64() {            // splitmix64
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double from_bits(uint64_t b) { double x; memcpy(&x, &b, 8); return x; }
static bool same_bits(double a, double b) { return memcmp(&a, &b, 8) == 0; }

int main() {
    std::vector<double> v = {0.0, from_bits(1), DBL_MIN, 1e-300, 1e-150, 1e-6, 0.5, 1.0, 2.0, 1e150, 1e300,
                             DBL_MAX, INFINITY};
    for (int i = 0; i < 4000; ++i) {
        v.push_back(from_bits(next_u64() & 0x7FEFFFFFFFFFFFFFull));          // any finite non-negative
        v.push_back(std::ldexp((double)(next_u64() >> 11), -53 - (int)(next_u64() % 64)));   // near 0 .. 1
    }
    long bad = 0, n = 0;
    for (size_t i = 0; i < v.size(); ++i) {
        for (size_t j = i % 7; j < v.size(); j += 7) {
            const double a = v[i], b = v[j];
            ++n;
            if (!same_bits(nn_max(a, b), fmax(a, b)) && a != b) ++bad;
            if (!same_bits(nn_min(a, b), fmin(a, b)) && a != b) ++bad;
            if (nn_less(a, b) != (a < b)) ++bad;
            if (nn_less(a, -b) != (a < -b)) ++bad;                         // a negative bound
        }
    }
    const double probes[] = {-1.0, -0.0, 0.0, 1e-200, 1e-150, 2e-150, 1.0, 1e149, 1e150, 1e151, -1e150,
                             INFINITY, -INFINITY, NAN, -NAN};
    for (double a : probes) {
        n += 2;
        if (in_range(a, 1e-150, 1e150) != (a > 1e-150 && a < 1e150)) ++bad;
        if (positive_bits(a) != (a > 0.0)) ++bad;
    }
    printf("%ld mismatches in %ld comparisons\n", bad, n);
    return bad ? 1 : 0;
}
