// Shared-memory FFT building blocks: power-of-two complex transforms of many rows at once,
// as Stockham stages of radix 16 (and one stage of radix 2, 4 or 8 for the remaining factor)
// whose butterflies run in registers.
//
// A stage of radix Q after sub-transforms of length m (m = product of the earlier radices)
// takes, for each j < L / Q, the Q values x[j + i L / Q], multiplies value i by
// exp(-+2 pi i i (j mod m) / (m Q)), transforms them with a Q-point DFT and writes output i to
// (j - j mod m) Q + j mod m + i m: natural order in and out, no bit reversal.  The Q-point
// DFTs split into radix-4 and radix-2 butterflies with their twiddles as constants.
//
// Rows sit in shared memory with one pad slot per 16 complex values (index i -> i + i / 16),
// which keeps the stride-16 accesses of the first stage free of bank conflicts, at an odd row
// stride (row_stride).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <vector>

namespace scola {
namespace fft {

__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded(int L) { return L + L / 16; }
// Row stride (complex values) of the rows of one transform batch: padded(L), made odd (a
// stride that is a multiple of the bank count would put a column of consecutive rows in one
// bank; strides tuned per access pattern measured no faster).  R, the rows per batch, is
// kept in the signature for the callers' buffer sizing.
__host__ __device__ constexpr int row_stride(int L, int R) { return (void)R, padded(L) | 1; }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {   // a conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// cos and sin of 2 pi e / 16
__device__ __forceinline__ float c16(int e) {
    constexpr float t[16] = {1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                             0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
                             -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
                             0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f};
    return t[e & 15];
}
__device__ __forceinline__ float s16(int e) { return c16(e - 4); }

// v * exp(SIGN 2 pi i e / 16), e a compile-time constant after unrolling
template <int SIGN>
__device__ __forceinline__ float2 w16(float2 v, int e) {
    const float c = c16(e), s = SIGN * s16(e);
    return make_float2(v.x * c - v.y * s, v.x * s + v.y * c);
}

// In-register DFTs, X_k = sum_n v_n exp(SIGN 2 pi i n k / Q), natural order in and out.
template <int SIGN>
__device__ __forceinline__ void dft2(float2 *v) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <int SIGN>
__device__ __forceinline__ void dft4(float2 &v0, float2 &v1, float2 &v2, float2 &v3) {
    const float2 t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3), d = csub(v1, v3);
    const float2 t3 = make_float2(-SIGN * d.y, SIGN * d.x);     // SIGN i (v1 - v3)
    v0 = cadd(t0, t2);
    v2 = csub(t0, t2);
    v1 = cadd(t1, t3);
    v3 = csub(t1, t3);
}

template <int SIGN>
__device__ __forceinline__ void dft4(float2 *v) { dft4<SIGN>(v[0], v[1], v[2], v[3]); }

// dft8 and dft16 leave output k in register slot perm<Q>(k) (a fixed transposition, so that
// each column of the two-level split is overwritten by its own results).
template <int SIGN>
__device__ __forceinline__ void dft8(float2 *v) {
    // n = n1 + 2 n2, k = k1 + 4 k2: X[k1 + 4 k2] = sum_n1 W2^(n1 k2) W8^(n1 k1) DFT4_n2(v[n1 + 2 n2])[k1];
    // the inner transforms leave (n1, k1) in slot n1 + 2 k1, X[k1 + 4 k2] goes to slot k2 + 2 k1
    dft4<SIGN>(v[0], v[2], v[4], v[6]);
    dft4<SIGN>(v[1], v[3], v[5], v[7]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        const float2 e = v[2 * k1], o = w16<SIGN>(v[2 * k1 + 1], 2 * k1);
        v[2 * k1] = cadd(e, o);
        v[2 * k1 + 1] = csub(e, o);
    }
}

template <int SIGN>
__device__ __forceinline__ void dft16(float2 *v) {
    // n = n1 + 4 n2, k = k1 + 4 k2: X[k1 + 4 k2] = sum_n1 W4^(n1 k2) W16^(n1 k1) DFT4_n2(v[n1 + 4 n2])[k1];
    // the inner transforms leave (n1, k1) in slot n1 + 4 k1, X[k1 + 4 k2] goes to slot k2 + 4 k1
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) dft4<SIGN>(v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
#pragma unroll
        for (int n1 = 1; n1 < 4; ++n1) v[n1 + 4 * k1] = w16<SIGN>(v[n1 + 4 * k1], n1 * k1);
        dft4<SIGN>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    }
}

template <int Q>
__host__ __device__ constexpr int perm(int k) {
    return Q == 16 ? (k >> 2) + 4 * (k & 3) : Q == 8 ? (k >> 2) + 2 * (k & 3) : k;
}

template <int Q, int SIGN>
__device__ __forceinline__ void dft(float2 *v) {
    if constexpr (Q == 2) dft2<SIGN>(v);
    if constexpr (Q == 4) dft4<SIGN>(v);
    if constexpr (Q == 8) dft8<SIGN>(v);
    if constexpr (Q == 16) dft16<SIGN>(v);
}

// Twiddles of a radix-16 stage after sub-transforms of length 16 (the same for every L):
// w256[16 i + k] = exp(-2 pi i i k / 256), i, k < 16; thread k reads w256[16 i + k], a
// contiguous run, where tw[i k L / 256] would be a stride-i (bank-conflicted) one.
constexpr int kW256 = 256;

// Whether a transform of length 2^logL reads tw at all: a radix-16 stage after sub-transforms
// of 256, or a last radix-2/4/8 stage after a radix-16 one (the first stage has no twiddles,
// the second radix-16 stage reads w256).
__host__ __device__ constexpr bool needs_tw(int logL) { return logL / 4 >= 3 || (logL % 4 != 0 && logL / 4 >= 1); }

// The w256 table (host, FP64 then rounded): 512 floats, re/im interleaved.
inline void append_w256(std::vector<float> &arena) {
    for (int i = 0; i < 16; ++i)
        for (int k = 0; k < 16; ++k) {
            const double a = -2.0 * 3.14159265358979323846 * (double)(i * k) / 256.0;
            arena.push_back((float)std::cos(a));
            arena.push_back((float)std::sin(a));
        }
}

// One Stockham stage of radix Q over `rows` rows of length L = 2^logL, after sub-transforms
// of length m: input element n of row r comes from load(r, n), output goes to the padded row
// r of dst (row stride padded(L)).  tw[e] = exp(-2 pi i e / L), e < L; w256 as above.
template <int Q, int SIGN, class Load>
__device__ __forceinline__ void stage(Load load, float2 *dst, int rows, int logL, int m, const float2 *tw,
                                      const float2 *w256) {
    constexpr int logQ = Q == 2 ? 1 : Q == 4 ? 2 : Q == 8 ? 3 : 4;
    const int L = 1 << logL, nb = L >> logQ, lognb = logL - logQ;
    const int Ls = row_stride(L, rows);
    const int step = L / (m * Q);
    for (int q = threadIdx.x; q < rows * nb; q += blockDim.x) {
        const int r = q >> lognb, j = q & (nb - 1);
        const int k = j & (m - 1);
        float2 *y = dst + r * Ls;
        float2 v[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) v[i] = load(r, j + i * nb);
        if (m > 1) {
            const bool w16 = Q == 16 && m == 16;
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                float2 t = w16 ? w256[16 * i + k] : tw[i * k * step];
                if (SIGN > 0) t.y = -t.y;
                v[i] = cmul(v[i], t);
            }
        }
        dft<Q, SIGN>(v);
        const int o = (j - k) * Q + k;
#pragma unroll
        for (int i = 0; i < Q; ++i) y[pad(o + i * m)] = v[perm<Q>(i)];
    }
}

struct NoHook {
    __device__ void operator()() const {}
};

// The whole transform of `rows` rows (SIGN -1 forward, +1 inverse, unnormalised).  The first
// stage reads through first(r, n) and writes dst; later stages ping-pong between dst and spare
// (first may read spare, never dst).  Returns the buffer holding the result; synchronises the
// block after every stage and calls after_first() once the first stage's barrier has passed
// (whatever first read is free from then on).  logL >= 1.
template <int SIGN, class Load, class Hook = NoHook>
__device__ float2 *transform(Load first, float2 *dst, float2 *spare, int rows, int logL, const float2 *tw,
                             const float2 *w256, Hook after_first = Hook()) {
    const int Ls = row_stride(1 << logL, rows);
    auto from = [&](const float2 *src) {
        return [src, Ls](int r, int n) { return src[r * Ls + pad(n)]; };
    };
    int m = 1, left = logL;
    float2 *a = dst, *b = spare;      // a: the next stage's output
    bool started = false;
    while (left >= 4) {
        if (!started) stage<16, SIGN>(first, a, rows, logL, m, tw, w256);
        else stage<16, SIGN>(from(b), a, rows, logL, m, tw, w256);
        __syncthreads();
        if (!started) after_first();
        started = true;
        float2 *t = a;
        a = b;
        b = t;
        m <<= 4;
        left -= 4;
    }
    if (left > 0) {
        if (!started) {
            if (left == 1) stage<2, SIGN>(first, a, rows, logL, m, tw, w256);
            if (left == 2) stage<4, SIGN>(first, a, rows, logL, m, tw, w256);
            if (left == 3) stage<8, SIGN>(first, a, rows, logL, m, tw, w256);
        } else {
            if (left == 1) stage<2, SIGN>(from(b), a, rows, logL, m, tw, w256);
            if (left == 2) stage<4, SIGN>(from(b), a, rows, logL, m, tw, w256);
            if (left == 3) stage<8, SIGN>(from(b), a, rows, logL, m, tw, w256);
        }
        __syncthreads();
        if (!started) after_first();
        float2 *t = a;
        a = b;
        b = t;
    }
    return b;
}

}  // namespace fft
}  // namespace scola
