// Seeded Gaussian random vectors for the cross-polytope hashes (Section 2.2:
// every coordinate of every r_i is drawn from N(0, 1)).
//
// Counter-based SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) feeds the
// cosine branch of the Box-Muller transform (Box and Muller, 1958):
//   stream id      s = 2 t + j                (table t, hash j)
//   initial state  seed XOR (0x9E3779B97F4A7C15 * (s + 1))   (mod 2^64)
//   output number  k of a stream = mix(state + (k + 1) * 0x9E3779B97F4A7C15)
//   coordinate     (i, c) uses outputs 2(i d + c) and 2(i d + c) + 1 as
//                  u1 = (top53 + 1) / 2^53 in (0, 1], u2 = top53 / 2^53,
//                  z = sqrt(-2 ln u1) cos(2 pi u2), rounded to FP32 and
//                  then to BF16 (nearest, ties to even).
// The paper only asks for N(0, 1) coordinates; keeping them on the BF16 grid
// (8 significant bits) leaves the vectors just as random for the hash and
// makes every projection q^T r an exact sum of three BF16 tensor-core
// products (q split into three BF16 pieces, r one piece).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/fpp.h"

namespace fpp {

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

// FP32 -> nearest BF16 (ties to even), returned as FP32; z is finite.
inline float round_to_bf16(float z) {
  uint32_t u;
  std::memcpy(&u, &z, 4);
  u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
  std::memcpy(&z, &u, 4);
  return z;
}

inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void fill_stream(uint64_t seed, int64_t stream, int64_t count, float* out) {
  const uint64_t s0 = seed ^ (kGolden * (uint64_t)(stream + 1));
  for (int64_t e = 0; e < count; ++e) {
    const uint64_t r1 = mix64(s0 + (uint64_t)(2 * e + 1) * kGolden);
    const uint64_t r2 = mix64(s0 + (uint64_t)(2 * e + 2) * kGolden);
    const double u1 = ((double)(r1 >> 11) + 1.0) / 9007199254740992.0;
    const double u2 = (double)(r2 >> 11) / 9007199254740992.0;
    const double z = std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    out[e] = round_to_bf16((float)z);
  }
}

}  // namespace

void generate_rotations(uint64_t seed, int L, int D, int d, float* R) {
  const int64_t per = (int64_t)D * d;
  const int streams = 2 * L;
  unsigned nth = std::thread::hardware_concurrency();
  if (nth == 0) nth = 1;
  if (nth > 32) nth = 32;
  if ((int64_t)streams * per < (1 << 16)) nth = 1;
  std::vector<std::thread> pool;
  for (unsigned w = 0; w < nth; ++w) {
    pool.emplace_back([=]() {
      for (int s = (int)w; s < streams; s += (int)nth) fill_stream(seed, s, per, R + (int64_t)s * per);
    });
  }
  for (auto& th : pool) th.join();
}

}  // namespace fpp
