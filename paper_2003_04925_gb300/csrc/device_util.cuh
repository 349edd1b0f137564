// Device helpers shared by the kernels.
#pragma once

#include "internal.h"

namespace scola {

// The padded PM grid of a box has P = 2 N_ghost = FDA order ghost layers on every side
// (padded index pc = c + P, S = Ng + 2P cells per axis).

// Number of padded cells outside the interior: (Ng+2P)^3 - Ng^3.
__host__ __device__ inline long long shell_count(int Ng, int P) {
    const long long a = Ng + 2 * P;
    return a * a * a - (long long)Ng * Ng * Ng;
}

// Padded coordinates (0..Ng+2P-1 per axis) of shell cell `idx`.  Enumeration: the 2P
// full i-planes {0..P-1, Ng+P..Ng+2P-1}; then, for interior i, the 2P full j-rows; then,
// for interior i and j, the 2P k-cells.  (32-bit arithmetic: a shell of Ng <= 256, P <= 6
// has fewer than 2^22 cells.)
__device__ inline void shell_coord(long long idx64, int Ng, int P, int &pi, int &pj, int &pk) {
    int idx = (int)idx64;
    const int S = Ng + 2 * P;
    const int plane = S * S;
    const int A = 2 * P * plane;
    if (idx < A) {
        const int q = idx / plane;
        const int r = idx - q * plane;
        pi = q < P ? q : Ng + q;
        pj = r / S;
        pk = r - pj * S;
        return;
    }
    idx -= A;
    const int rowblk = 2 * P * S;
    const int B = Ng * rowblk;
    if (idx < B) {
        pi = P + idx / rowblk;
        const int r = idx - (pi - P) * rowblk;
        const int q = r / S;
        pj = q < P ? q : Ng + q;
        pk = r - q * S;
        return;
    }
    idx -= B;
    const int line = 2 * P * Ng;
    pi = P + idx / line;
    const int r = idx - (pi - P) * line;
    pj = P + r / (2 * P);
    const int q = r - (pj - P) * (2 * P);
    pk = q < P ? q : Ng + q;
}

// Central-difference coefficients of FDA order 2, 4, 6 (N_ghost = order / 2 terms):
// gradient f' = (1/d) sum_m g_m (f_{+m} - f_{-m}); second derivative
// f'' = (1/d^2) (s_0 f + sum_m s_m (f_{+m} + f_{-m})).
template <int ORDER> struct Fda;
template <> struct Fda<2> {
    static constexpr int ng = 1;
    __device__ static float g(int m) { return 0.5f; }
    __device__ static float s(int m) { return m == 0 ? -2.0f : 1.0f; }
};
template <> struct Fda<4> {
    static constexpr int ng = 2;
    __device__ static float g(int m) { return m == 1 ? 2.0f / 3.0f : -1.0f / 12.0f; }
    __device__ static float s(int m) { return m == 0 ? -2.5f : (m == 1 ? 4.0f / 3.0f : -1.0f / 12.0f); }
};
template <> struct Fda<6> {
    static constexpr int ng = 3;
    __device__ static float g(int m) { return m == 1 ? 0.75f : (m == 2 ? -0.15f : 1.0f / 60.0f); }
    __device__ static float s(int m) {
        return m == 0 ? -49.0f / 18.0f : (m == 1 ? 1.5f : (m == 2 ? -0.15f : 1.0f / 90.0f));
    }
};

// Boundary term of Eq. 62 for the interior cell (i, j, k): the order-n Laplacian's
// contributions of the Dirichlet values in the ghost layers (unscaled by 1/dg^2).  P_c is
// the padded potential at the cell; S the padded row length.  Per axis: the offsets m
// that reach past the lower face (m > x) and past the upper face (m >= Ng - x).
template <int ORDER>
__device__ __forceinline__ float boundary_term_n(const float *P_c, int i, int j, int k, int Ng, int S) {
    float bc = 0.0f;
    const int st[3] = {S * S, S, 1};
    const int x[3] = {i, j, k};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int m = 1; m <= Fda<ORDER>::ng; ++m) {
            if (m > x[a]) bc += Fda<ORDER>::s(m) * P_c[-m * st[a]];
            if (m >= Ng - x[a]) bc += Fda<ORDER>::s(m) * P_c[m * st[a]];
        }
    }
    return bc;
}

__device__ __forceinline__ float boundary_term(const float *P_c, int i, int j, int k, int Ng, int S, int order) {
    return order == 2 ? boundary_term_n<2>(P_c, i, j, k, Ng, S)
                      : (order == 4 ? boundary_term_n<4>(P_c, i, j, k, Ng, S) : boundary_term_n<6>(P_c, i, j, k, Ng, S));
}

__device__ __forceinline__ void decode_local(int local, int n, int &i, int &j, int &k) {
    k = local % n;
    const int t = local / n;
    j = t % n;
    i = t / n;
}

// Per-tile final scale factors: box b's FP32 coefficients at force evaluation k (see Ctx::coef),
// or null when the launch uses uniform scalars.
__device__ __forceinline__ const float *box_coef(const float *coef, int box, int k, int nk) {
    return coef ? coef + ((long long)box * nk + k) * 8 : nullptr;
}

// Sorted deposit: the interior mesh of a box is cut into bricks of kBrick^3 cells.
constexpr int kBrick = 16;

struct SortEntry {
    int key;          // box-local key ((bx nbe + by) nbe + bz) 8 + class, or -1 (no weight inside)
    float4 e;         // f_x, f_y, f_z, packed i0 (+2, 10 bits per axis)
};

// The sorted deposit's key and entry of a particle at box-local lattice index b with
// displacement s: the clamped mesh coordinate u (as in the CIC deposit) has integer part
// i0 and fractions f; the key is the brick of the upper corner i0 + 1 with a 3-bit class
// whose bit a says that the lower corner lies in the brick below along axis a.  The count
// pass (in the kick-drift of the previous step, or its own kernel) and the fill pass
// compute it with this one function from the same FP32 values.
__device__ __forceinline__ SortEntry brick_entry(const BoxDesc &B, const float (&s)[3], const int (&b)[3]) {
    const int Ng = B.Ng, nbe = B.nbe;
    int i0[3];
    float f[3];
    bool inside = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float u = fmaf(s[a], B.inv_dg, fmaf((float)b[a], B.q2u, 0.5f * B.q2u - 0.5f));
        u = fminf(fmaxf(u, -2.0f), (float)Ng + 1.0f);
        const float fl = floorf(u);
        i0[a] = (int)fl;
        f[a] = u - fl;
        inside = inside && i0[a] >= -1 && i0[a] < Ng;
    }
    SortEntry r;
    r.key = -1;
    r.e = make_float4(f[0], f[1], f[2],
                      __int_as_float((i0[0] + 2) | ((i0[1] + 2) << 10) | ((i0[2] + 2) << 20)));
    if (inside) {
        const int cls = (((i0[0] + 1) & (kBrick - 1)) == 0 ? 1 : 0) | (((i0[1] + 1) & (kBrick - 1)) == 0 ? 2 : 0) |
                        (((i0[2] + 1) & (kBrick - 1)) == 0 ? 4 : 0);
        r.key = ((((i0[0] + 1) >> 4) * nbe + ((i0[1] + 1) >> 4)) * nbe + ((i0[2] + 1) >> 4)) * 8 + cls;
    }
    return r;
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
        const int num = (2 * (pc[a] - B.gpad) + 1) * B.Nsc - B.Ng;
        int q = num / den, r = num - q * den;
        if (r < 0) {
            r += den;
            --q;
        }
        i0[a] = t[a] * Ntile - B.Nbuf + q;
        f[a] = (float)r / (float)den;
    }
}

// The same stencil with the offsets in FP64, for the FP64 accumulation of the C.3 shell: the
// exact integer r times the box's FP64 reciprocal of den (two FP64 roundings, far below the
// FP32 rounding of the result; FP64 division is slow on this GPU).
__device__ __forceinline__ void shell_stencil_d(const BoxDesc &B, const int pc[3], int Ntile, int i0[3],
                                                double f[3]) {
    const int t[3] = {B.tx, B.ty, B.tz};
    const int den = 2 * B.Ng;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int num = (2 * (pc[a] - B.gpad) + 1) * B.Nsc - B.Ng;
        int q = num / den, r = num - q * den;
        if (r < 0) {
            r += den;
            --q;
        }
        i0[a] = t[a] * Ntile - B.Nbuf + q;
        f[a] = (double)r * B.inv_2ng_d;
    }
}

__device__ __forceinline__ int wrap(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

}  // namespace scola
