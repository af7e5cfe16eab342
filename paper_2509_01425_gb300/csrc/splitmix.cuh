// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014; public-domain reference by
// S. Vigna): the state advances by GAMMA and each output passes the state
// through the finaliser below. first_output(k) is the first output of a
// generator whose state is k.
#pragma once
#include <stdint.h>

namespace hicr {

static constexpr uint64_t SM64_GAMMA = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t sm64_finalise(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t sm64_first_output(uint64_t k) {
  return sm64_finalise(k + SM64_GAMMA);
}

}  // namespace hicr
