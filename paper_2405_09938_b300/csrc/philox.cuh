// Counter-based random numbers for the echo path: Philox4x32-10 (Salmon, Moraes,
// Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11), written
// from the published round function and key schedule, usable on host and device.
//
// Streams: counter (id, 0, word2, 0) with key (seed_lo, seed_hi ^ stream).
//   speckle   : id = facet, word2 = coherence epoch, stream 0
//   wave phase: id = component, word2 = 0 (homogeneous sea state) or 1 + corner
//               index (tile of a heterogeneous sea state), stream 0x57415645
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define HARM_HD __host__ __device__ __forceinline__
#else
#define HARM_HD inline
#endif

namespace harm {

constexpr uint32_t kStreamSpeckle = 0x00000000u;
constexpr uint32_t kStreamWave = 0x57415645u;

struct U32x4 {
    uint32_t x, y, z, w;
};

HARM_HD void mulhilo32(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo)
{
#ifdef __CUDA_ARCH__
    lo = a * b;
    hi = __umulhi(a, b);
#else
    uint64_t p = (uint64_t)a * (uint64_t)b;
    lo = (uint32_t)p;
    hi = (uint32_t)(p >> 32);
#endif
}

// Ten rounds; the key advances by the Weyl constants between rounds.
HARM_HD U32x4 philox4x32_10(U32x4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, c.x, hi0, lo0);
        mulhilo32(0xCD9E8D57u, c.z, hi1, lo1);
        U32x4 o;
        o.x = hi1 ^ c.y ^ k0;
        o.y = lo1;
        o.z = hi0 ^ c.w ^ k1;
        o.w = lo0;
        c = o;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

HARM_HD U32x4 philox_stream(uint64_t seed, uint32_t stream, uint32_t id, uint32_t word2)
{
    U32x4 c{id, 0u, word2, 0u};
    return philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) ^ stream);
}

}  // namespace harm
