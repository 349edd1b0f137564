// Device self-test of the fixed-point conversions used by the CIC deposits: the 32-bit
// forms in device_util.cuh against CUDA's direct 64-bit conversions, on generated inputs.
#include "device_util.cuh"

namespace scola {

namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    // splitmix64 finaliser (Steele, Lea and Flood 2014)
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Input i: a weight in [0, 1] (uniform, near 0, near 1, exactly 0 or 1) and a 64-bit
// count (random magnitude, or a pattern that sits exactly on a float rounding tie).
__global__ void k_selftest(long long n, unsigned long long seed, unsigned long long *mismatch) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long r = mix64(seed ^ mix64((unsigned long long)i));
        const unsigned r32 = (unsigned)r;
        float w;
        switch ((r >> 32) & 7) {
            case 0: w = 0.0f; break;
            case 1: w = 1.0f; break;
            case 2: w = __uint_as_float(0x3F800000u - 1u - (r32 & 0xFFFFu)); break;   // just below 1
            case 3: w = __uint_as_float(0x2F800000u + (r32 & 0x00FFFFFFu)); break;     // ~2^-32
            default: w = (float)(r32 >> 8) * (1.0f / 16777216.0f); break;
        }
        if (weight_to_fixed(w) != __float2ull_rn(w * 4294967296.0f)) atomicAdd(mismatch, 1ull);
        unsigned long long x;
        const int sh = (int)((r >> 35) & 63);
        if ((r >> 41) & 1) {
            // a tie: 24 significant bits, then exactly half an ulp, at a random position
            const unsigned long long m = ((r >> 42) & 0x7FFFFFull) | 0x800000ull;   // 24 bits
            const int s2 = sh % 40;                                                 // 25 + 39 <= 64 bits
            x = ((m << 1) | 1ull) << s2;
            if (((r >> 40) & 1) && s2 > 0) x |= 1ull;   // just above the tie
        } else {
            x = mix64(r) >> sh;
        }
        if (__float_as_uint(fixed_to_float(x)) != __float_as_uint(__ull2float_rn(x))) atomicAdd(mismatch, 1ull);
    }
}

}  // namespace

}  // namespace scola

extern "C" scola_status scola_selftest_conversions(int64_t n, uint64_t seed, int64_t *mismatches) {
    if (!mismatches || n < 0) return SCOLA_ERR_INVALID_ARG;
    unsigned long long *d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned long long)) != cudaSuccess) return SCOLA_ERR_OOM;
    cudaError_t e = cudaMemset(d, 0, sizeof(unsigned long long));
    if (e == cudaSuccess && n > 0) {
        scola::k_selftest<<<1024, 256>>>((long long)n, (unsigned long long)seed, d);
        e = cudaGetLastError();
    }
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return SCOLA_ERR_CUDA;
    *mismatches = (int64_t)h;
    return SCOLA_OK;
}
