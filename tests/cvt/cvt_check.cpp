// Host check of the integer binary64 <-> binary32 conversions (csrc/cvt.cuh) against the
// C++ conversions of this machine (IEEE 754 round to nearest, ties to even): random bit
// patterns over every exponent, and the edges (ties, the largest finite values, the
// subnormal ranges, zeros, infinities, NaNs). Prints the number of mismatches.
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <random>

#include "../../paper_2607_26382_b300/csrc/cvt.cuh"

static uint32_t b32(float x) { uint32_t b; std::memcpy(&b, &x, 4); return b; }
static uint64_t b64(double x) { uint64_t b; std::memcpy(&b, &x, 8); return b; }
static double d_of(uint64_t b) { double x; std::memcpy(&x, &b, 8); return x; }
static float f_of(uint32_t b) { float x; std::memcpy(&x, &b, 4); return x; }

static long long bad = 0, checked = 0;

static void check_narrow(double x)
{
    const float ref = (float)x, got = gf::f32_rn_of_f64(x);
    ++checked;
    if (std::isnan(ref) ? !std::isnan(got) : b32(ref) != b32(got)) {
        if (bad < 10) std::printf("narrow %a (%016llx): ref %08x got %08x\n", x, (unsigned long long)b64(x), b32(ref), b32(got));
        ++bad;
    }
}

static void check_widen(float x)
{
    const double ref = (double)x, got = gf::f64_of_f32(x);
    ++checked;
    if (std::isnan(ref) ? !std::isnan(got) : b64(ref) != b64(got)) {
        if (bad < 10) std::printf("widen %a (%08x): ref %016llx got %016llx\n", (double)x, b32(x), (unsigned long long)b64(ref), (unsigned long long)b64(got));
        ++bad;
    }
}

int main()
{
    std::mt19937_64 rng(20261204);
    // random bit patterns: every binary64 exponent equally often
    for (int i = 0; i < 4000000; ++i) {
        const uint64_t r = rng();
        const uint64_t e = rng() % 2048;
        check_narrow(d_of((r & 0x800fffffffffffffull) | (e << 52)));
    }
    // exponents near the binary32 range and its subnormals, low fraction bits at the ties
    for (int i = 0; i < 4000000; ++i) {
        const uint64_t r = rng();
        const uint64_t e = 850 + rng() % 330;   // 2^-173 .. 2^156
        uint64_t m = r & 0x000fffffffffffffull;
        const int mode = (int)(rng() % 4);
        if (mode == 1) m = (m & ~0x1fffffffull) | 0x10000000ull;   // a tie for normal results
        if (mode == 2) m = (m & ~0x1fffffffull) | 0x0fffffffull;   // just below a tie
        if (mode == 3) m = (m & ~0x1fffffffull) | 0x10000001ull;   // just above
        check_narrow(d_of((r & 0x8000000000000000ull) | (e << 52) | m));
    }
    // subnormal results: every shift, ties and their neighbours
    for (int e = 860; e <= 897; ++e)
        for (int i = 0; i < 20000; ++i) {
            const uint64_t m = rng() & 0x000fffffffffffffull;
            const int sh = 926 - e;
            uint64_t mm = m;
            if (sh < 64 && (i % 3) == 1) mm = (m & ~((1ull << (sh >= 53 ? 52 : sh)) - 1)) | ((sh >= 53 ? 0 : (1ull << (sh - 1))) & 0x000fffffffffffffull);
            check_narrow(d_of(((uint64_t)e << 52) | mm));
            check_narrow(-d_of(((uint64_t)e << 52) | mm));
        }
    const double edges[] = {0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 3.4028235677973366e38, 3.402823567797337e38,
                            3.4028236e38, 1e39, -1e39, INFINITY, -INFINITY, NAN, 1.1754943508222875e-38,
                            1.1754942807573643e-38, 1.401298464324817e-45, 7.006492321624085e-46,
                            7.006492321624087e-46, 2.1019476964872256e-45, 1e-46, 4.9e-324, -4.9e-324, 2.2250738585072014e-308};
    for (double x : edges) check_narrow(x);
    // widening: every binary32 exponent, subnormals, specials
    for (int i = 0; i < 4000000; ++i) check_widen(f_of((uint32_t)rng()));
    for (uint32_t m = 1; m < (1u << 23); m += 97) { check_widen(f_of(m)); check_widen(f_of(m | 0x80000000u)); }
    const float fedges[] = {0.0f, -0.0f, INFINITY, -INFINITY, NAN, 1.17549435e-38f, 1.4e-45f, 3.40282347e38f};
    for (float x : fedges) check_widen(x);
    std::printf("checked %lld mismatches %lld\n", checked, bad);
    return bad != 0;
}
