// Bit-sliced counting: 32 independent per-dimension counters held in the bit
// positions of a few uint32 planes (plane k holds bit k of every count), so
// one logic operation advances 32 counters.  Used by the Level-ID majority
// (k_levelid.cu) and the class-grouped bit counts of training (k_train.cu).
#pragma once

#include <cstdint>

namespace hdc {
namespace {

// Full adder per bit position: l = a ^ b ^ c (weight 1), h = majority
// (weight 2); each a single three-input logic operation.
__device__ __forceinline__ void csa(uint32_t &h, uint32_t &l, uint32_t a, uint32_t b, uint32_t c)
{
    h = (a & b) | (a & c) | (b & c);
    l = a ^ b ^ c;
}

// Add 16 rows of weight 1 to the carry-save state c1, c2, c4, c8 (planes of
// weight 1, 2, 4, 8) with a tree of 15 full adders; returns the row of
// weight 16 that carries out of c8.
__device__ __forceinline__ uint32_t csa16(uint32_t &c1, uint32_t &c2, uint32_t &c4, uint32_t &c8,
                                          const uint32_t (&r)[16])
{
    uint32_t a2, b2, a4, b4, a8, b8, e16;
    csa(a2, c1, c1, r[0], r[1]);
    csa(b2, c1, c1, r[2], r[3]);
    csa(a4, c2, c2, a2, b2);
    csa(a2, c1, c1, r[4], r[5]);
    csa(b2, c1, c1, r[6], r[7]);
    csa(b4, c2, c2, a2, b2);
    csa(a8, c4, c4, a4, b4);
    csa(a2, c1, c1, r[8], r[9]);
    csa(b2, c1, c1, r[10], r[11]);
    csa(a4, c2, c2, a2, b2);
    csa(a2, c1, c1, r[12], r[13]);
    csa(b2, c1, c1, r[14], r[15]);
    csa(b4, c2, c2, a2, b2);
    csa(b8, c4, c4, a4, b4);
    csa(e16, c8, c8, a8, b8);
    return e16;
}

}  // namespace
}  // namespace hdc
