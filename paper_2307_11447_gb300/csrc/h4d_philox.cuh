// h4d_philox.cuh -- the counter-based random stream of libh4d (device side).
// Philox4x64-10 (Salmon, Moraes, Dror and Shaw, SC'11): counter {c0, c1, purpose, 0},
// key {seed, replica}; every draw has a fixed address, so results do not depend on
// thread scheduling.
#pragma once
#include <cstdint>

namespace h4d {

typedef unsigned long long u64;

// purposes; training minibatches use key {seed, kTrainKey}, disjoint from every replica
enum : u64 { kPurTrial = 1, kPurGamma = 2, kPurThermo = 3, kPurVinit = 4, kPurTrain = 5 };
constexpr u64 kTrainKey = 0x8000000000000000ULL;

__device__ __forceinline__ void philox4x64(u64 c[4], u64 k0, u64 k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const u64 m0 = 0xD2E7470EE14C6C93ULL, m1 = 0xCA5A826395121157ULL;
    u64 lo0 = m0 * c[0], hi0 = __umul64hi(m0, c[0]);
    u64 lo1 = m1 * c[2], hi1 = __umul64hi(m1, c[2]);
    u64 n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B97F4A7C15ULL;
    k1 += 0xBB67AE8584CAA73BULL;
  }
}

__device__ __forceinline__ void draw4(u64 seed, u64 rep, u64 c0, u64 c1, u64 pur, u64 out[4]) {
  out[0] = c0; out[1] = c1; out[2] = pur; out[3] = 0;
  philox4x64(out, seed, rep);
}
__device__ __forceinline__ double u01(u64 r) { return (double)(r >> 11) * 0x1.0p-53; }
__device__ __forceinline__ double u01_open(u64 r) { return (double)((r >> 11) + 1) * 0x1.0p-53; }
__device__ __forceinline__ int pick_index(u64 r, int n) { return (int)(((r >> 32) * (u64)n) >> 32); }
__device__ __forceinline__ double gauss_c(u64 a, u64 b) {
  return sqrt(-2.0 * log(u01_open(a))) * cos(2.0 * 3.141592653589793 * u01(b));
}
__device__ __forceinline__ double gauss_s(u64 a, u64 b) {
  return sqrt(-2.0 * log(u01_open(a))) * sin(2.0 * 3.141592653589793 * u01(b));
}

}  // namespace h4d
