// Philox-4x32-10 counter-based random numbers (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
// as easy as 1, 2, 3", SC'11): ten rounds of the 4x32 Philox S-box on a 128-bit counter under a
// 64-bit key, with the Weyl key schedule.  Shared by the phase-space kernels (every event's random
// numbers depend only on seed, stream and event index) and the training-batch sampler.
#pragma once
#include <cstdint>

namespace {

__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t h0 = __umulhi(0xD2511F53u, c[0]), l0 = 0xD2511F53u * c[0];
    const uint32_t h1 = __umulhi(0xCD9E8D57u, c[2]), l1 = 0xCD9E8D57u * c[2];
    const uint32_t n0 = h1 ^ c[1] ^ k0, n2 = h0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = l1; c[2] = n2; c[3] = l0;
  }
}

// block `blk` of four words for event e: counter (e lo, blk, stream, e hi), key = seed
__device__ __forceinline__ void philox_block(uint64_t seed, uint32_t stream, uint64_t e, uint32_t blk, uint32_t w[4]) {
  w[0] = (uint32_t)e; w[1] = blk; w[2] = stream; w[3] = (uint32_t)(e >> 32);
  philox10(w, (uint32_t)seed, (uint32_t)(seed >> 32));
}

}  // namespace
