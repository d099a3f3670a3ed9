// Morton key arithmetic of the hierarchically sorted order (Sec. 3.1): 21 bits per axis of the
// unit box, interleaved with x owning the highest bit of each level triple.
#pragma once

#include "f64bits.cuh"

__device__ __forceinline__ unsigned long long spread3(unsigned int v)
{
    // place the 21 bits of v at every third bit position
    unsigned long long x = v & 0x1fffffull;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// floor(v 2^21) clamped to the 21-bit range, from the bits of v (no FP64 instruction)
__device__ __forceinline__ unsigned int quantise21(double v) { return fmm_quantise21(v); }
