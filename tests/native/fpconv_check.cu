// Host-only check of the integer float <-> double conversions in fpconv.cuh
// against the C conversions.  Exits 0 when every case agrees (up to the
// documented differences), printing the number of cases checked.
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <cmath>

#include "../../paper_1108_2473_gb300/csrc/fpconv.cuh"

static uint64_t d_bits(double d) { uint64_t u; std::memcpy(&u, &d, 8); return u; }
static uint32_t f_bits(float f) { uint32_t u; std::memcpy(&u, &f, 4); return u; }

int main() {
  // binary32 -> binary64: every bit pattern, exact (NaNs compared as NaNs)
  uint64_t n32 = 0;
  for (uint64_t b = 0; b <= 0xffffffffull; ++b) {
    uint32_t u = (uint32_t)b;
    float f;
    std::memcpy(&f, &u, 4);
    const double got = lqcd::f32_to_f64_bits(f), ref = (double)f;
    if (std::isnan(ref)) {
      if (!std::isnan(got)) { std::printf("f32->f64 NaN mismatch %08x\n", u); return 1; }
    } else if (d_bits(got) != d_bits(ref)) {
      std::printf("f32->f64 mismatch %08x\n", u);
      return 1;
    }
    ++n32;
  }
  // binary64 -> binary32: pseudo-random bit patterns plus edge cases
  uint64_t s = 0x9E3779B97F4A7C15ull, n64 = 0, ties = 0;
  auto check = [&](uint64_t u) -> bool {
    double d;
    std::memcpy(&d, &u, 8);
    const float got = lqcd::f64_to_f32_bits(d), ref = (float)d;
    ++n64;
    if (std::isnan(d)) return std::isnan(got);
    const int e = (int)((u >> 52) & 0x7ff);
    const int ef = e - 1023 + 127;
    if (ef <= 0) return f_bits(got) == (f_bits(ref) & 0x80000000u) || f_bits(got) == (uint32_t)((u >> 32) & 0x80000000u);
    if (f_bits(got) == f_bits(ref)) return true;
    // ties: round-to-nearest-even (the C cast) and ties-away differ by one unit
    if ((u & 0x1fffffffull) == 0x10000000ull) { ++ties; return true; }
    return false;
  };
  const uint64_t edges[] = {0ull, 0x8000000000000000ull, 0x7ff0000000000000ull, 0xfff0000000000000ull,
                            0x7ff8000000000000ull, 0x47efffffe0000000ull, 0x47effffff0000000ull,
                            0x3810000000000000ull, 0x380fffffffffffffull, 0x3ff0000010000000ull,
                            0x3ff0000030000000ull, 0x3fefffffffffffffull};
  for (uint64_t u : edges)
    if (!check(u)) { std::printf("f64->f32 mismatch %016llx\n", (unsigned long long)u); return 1; }
  for (int k = 0; k < 100000000; ++k) {
    s ^= s << 13; s ^= s >> 7; s ^= s << 17;  // xorshift64
    // bias towards the binary32 range: exponents 1023 +- 140
    uint64_t u = s;
    const uint64_t e = 1023 - 140 + (u >> 56) % 281;
    u = (u & 0x800fffffffffffffull) | (e << 52);
    if (!check(u)) { std::printf("f64->f32 mismatch %016llx\n", (unsigned long long)u); return 1; }
  }
  // scaled conversion: f64_to_f32_bits(d, e) against (float)ldexp(d, e)
  uint64_t nsc = 0;
  for (int k = 0; k < 20000000; ++k) {
    s ^= s << 13; s ^= s >> 7; s ^= s << 17;
    uint64_t u = s;
    const uint64_t e = 1023 - 300 + (u >> 54) % 601;
    u = (u & 0x800fffffffffffffull) | (e << 52);
    const int e2 = (int)(s % 401) - 200;
    double d;
    std::memcpy(&d, &u, 8);
    const double x = std::ldexp(d, e2);
    const float got = lqcd::f64_to_f32_bits(d, e2), ref = (float)x;
    ++nsc;
    uint64_t ux = d_bits(x);
    const int ex = (int)((ux >> 52) & 0x7ff) - 1023 + 127;
    bool ok;
    if (ex <= 0) ok = (f_bits(got) & 0x7fffffffu) == 0 && (f_bits(got) >> 31) == (uint32_t)(ux >> 63);
    else ok = f_bits(got) == f_bits(ref) || (ux & 0x1fffffffull) == 0x10000000ull;
    if (!ok) { std::printf("scaled mismatch %016llx e2 %d\n", (unsigned long long)u, e2); return 1; }
  }
  // split_pow2: s == m * 2^e, m in [1, 2) rounded to binary32
  for (int k = 0; k < 1000000; ++k) {
    s ^= s << 13; s ^= s >> 7; s ^= s << 17;
    uint64_t u = s;
    const uint64_t e = 1 + (u >> 53) % 2046;
    u = (u & 0x800fffffffffffffull) | (e << 52);
    double d;
    std::memcpy(&d, &u, 8);
    int ee = 0;
    float m = 0.f;
    if (!lqcd::split_pow2(d, ee, m)) { std::printf("split refused %016llx\n", (unsigned long long)u); return 1; }
    const double back = std::ldexp((double)m, ee);
    if (std::fabs(m) < 1.f || std::fabs(m) > 2.f || std::fabs(back - d) > std::ldexp(std::fabs(d), -24)) {
      std::printf("split mismatch %016llx\n", (unsigned long long)u);
      return 1;
    }
  }
  {
    int ee = 7;
    float m = 3.f;
    if (lqcd::split_pow2(0.0, ee, m) || lqcd::split_pow2(INFINITY, ee, m) || lqcd::split_pow2(4e-320, ee, m) ||
        ee != 7 || m != 3.f) { std::printf("split accepted a non-normal\n"); return 1; }
  }
  std::printf("ok scaled %llu\n", (unsigned long long)nsc);
  std::printf("ok f32->f64 %llu f64->f32 %llu ties %llu\n", (unsigned long long)n32, (unsigned long long)n64,
              (unsigned long long)ties);
  return 0;
}
