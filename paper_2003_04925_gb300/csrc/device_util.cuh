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

__device__ __forceinline__ int wrap(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

}  // namespace scola
