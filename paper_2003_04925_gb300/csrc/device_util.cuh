// Device helpers shared by the kernels.
#pragma once

#include "internal.h"

namespace scola {

// Number of padded cells outside the interior: (Ng+4)^3 - Ng^3.
__host__ __device__ inline long long shell_count(int Ng) {
    const long long a = Ng + 4;
    return a * a * a - (long long)Ng * Ng * Ng;
}

// Padded coordinates (0..Ng+3 per axis) of shell cell `idx`.  Enumeration:
// the four full i-planes {0, 1, Ng+2, Ng+3}; then, for interior i, the four
// full j-rows {0, 1, Ng+2, Ng+3}; then, for interior i and j, the four
// k-cells {0, 1, Ng+2, Ng+3}.
__device__ inline void shell_coord(long long idx, int Ng, int &pi, int &pj, int &pk) {
    const int S = Ng + 4;
    const long long plane = (long long)S * S;
    const long long A = 4 * plane;
    if (idx < A) {
        const int q = (int)(idx / plane);
        const long long r = idx - q * plane;
        pi = q < 2 ? q : Ng + q;
        pj = (int)(r / S);
        pk = (int)(r - (long long)pj * S);
        return;
    }
    idx -= A;
    const long long rowblk = 4LL * S;
    const long long B = (long long)Ng * rowblk;
    if (idx < B) {
        pi = 2 + (int)(idx / rowblk);
        const int r = (int)(idx % rowblk);
        const int q = r / S;
        pj = q < 2 ? q : Ng + q;
        pk = r - q * S;
        return;
    }
    idx -= B;
    pi = 2 + (int)(idx / (4LL * Ng));
    const int r = (int)(idx % (4LL * Ng));
    pj = 2 + r / 4;
    const int q = r & 3;
    pk = q < 2 ? q : Ng + q;
}

__device__ __forceinline__ void decode_local(int local, int n, int &i, int &j, int &k) {
    k = local % n;
    const int t = local / n;
    j = t % n;
    i = t / n;
}

// 2^-32 fixed-point value of a CIC weight w in [0, 1]: round-to-nearest of w 2^32 (the
// same integer as a direct float -> uint64 conversion), computed with 32-bit conversions
// only (64-bit integer conversions run on the FP64 pipe, which is narrow on this GPU).
__device__ __forceinline__ unsigned long long weight_to_fixed(float w) {
    const float v = w * 4294967296.0f;
    return v >= 4294967296.0f ? (1ull << 32) : (unsigned long long)__float2uint_rn(v);
}

// Correctly rounded float of a 64-bit count (round to nearest even, as a direct
// uint64 -> float conversion), from 32-bit operations: the top 32 significant bits with a
// sticky bit for the rest, converted once and scaled by an exact power of two.
__device__ __forceinline__ float fixed_to_float(unsigned long long x) {
    const unsigned hi = (unsigned)(x >> 32), lo = (unsigned)x;
    if (hi == 0) return __uint2float_rn(lo);
    const int lz = __clz(hi);
    const unsigned top = lz ? (hi << lz) | (lo >> (32 - lz)) : hi;
    const unsigned rest = lz ? lo << lz : lo;
    const float m = __uint2float_rn(top | (rest != 0u ? 1u : 0u));
    return m * __int_as_float((127 + 32 - lz) << 23);
}

// Trilinear stencil on the LPT grid (nodes at (i + 1/2) dq, N = Np) at the centre of padded
// mesh cell pc of a box (C.3): lower node i0 (not wrapped) and offsets f.  In node units the
// cell centre is u = (t Ntile - Nbuf) + ((2 pc - 3) Nsc - Ng) / (2 Ng), so i0 and the
// remainder are exact integers and f is one correctly rounded division.
__device__ __forceinline__ void shell_stencil(const BoxDesc &B, const int pc[3], int Ntile, int i0[3], float f[3]) {
    const int t[3] = {B.tx, B.ty, B.tz};
    const int den = 2 * B.Ng;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int num = (2 * pc[a] - 3) * B.Nsc - B.Ng;
        int q = num / den, r = num - q * den;
        if (r < 0) {
            r += den;
            --q;
        }
        i0[a] = t[a] * Ntile - B.Nbuf + q;
        f[a] = (float)r / (float)den;
    }
}

__device__ __forceinline__ int wrap(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

}  // namespace scola
