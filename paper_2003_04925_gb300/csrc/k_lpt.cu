// Full-box initial conditions and 2LPT (Sec. 3.1, steps A.1-A.2; Sec. 2.1, Eqs. 5-6).
//
// The Fourier transforms are cuFFT calls issued by the host (capi.cu); the
// spectral multiplications and the configuration-space operations are here.
// FDA order 2 throughout, spacing d = L/N:
//   colouring    delta^(k) = w^(k) sqrt(P(|k|) / d^3) / N^3, delta^(0) = 0 (the factor is
//                tabulated on the host in FP64 per integer |n|^2, stored FP32)
//   inverse Lap  phi^ = f^ / Lambda(k), Lambda = -(4/d^2) sum sin^2(pi n_i / N)
//   phi_,ij      = IFFT[-D_i D_j phi1^],  D_i = sin(2 pi n_i / N) / d
//                  (the central difference applied twice)
//   source       sum_{i>j} phi_,ii phi_,jj - phi_,ij^2
//   Psi          central-difference gradient at the grid nodes (periodic)
// The sine tables sin(pi n/N) and sin(2 pi n/N)/d are FP64 host values stored in FP32.
#include <cmath>

#include "device_util.cuh"

namespace scola {

namespace {

// the wrapped wavenumber of DFT index i: 0 .. (N - 1) / 2, then negative (-N / 2 first for even N)
__device__ __forceinline__ int wavenumber(int i, int N) { return 2 * i < N ? i : i - N; }

// White noise (step A.1) from Philox4x32-10 (Salmon et al. 2011): counter block g = (g mod
// 2^32, g div 2^32, 0, 0) under the key (seed mod 2^32, seed div 2^32); ten rounds that
// multiply words 0 and 2 by the round multipliers and mix the product halves with words 1
// and 3 and the key, the key bumped by the Weyl increments before every round after the
// first.  Each word's top 24 bits give the uniform (x + 1/2) 2^-24 (exact in FP32, in
// (0, 1)); words (0, 1) and (2, 3) become two standard normals each by Box-Muller:
// sqrt(-2 ln u0) (cos, sin)(2 pi u1).  Cell i takes word i % 4 of block i / 4.
constexpr unsigned kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr unsigned kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(unsigned c0, unsigned c1, unsigned k0, unsigned k1) {
    unsigned c2 = 0u, c3 = 0u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += kPhiloxW0;
            k1 += kPhiloxW1;
        }
        const unsigned hi0 = __umulhi(kPhiloxM0, c0), lo0 = kPhiloxM0 * c0;
        const unsigned hi1 = __umulhi(kPhiloxM1, c2), lo1 = kPhiloxM1 * c2;
        const unsigned n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ float unit_uniform(unsigned x) {
    return ((float)(x >> 8) + 0.5f) * 5.9604644775390625e-8f;   // 2^-24
}

__global__ void k_white_noise(float *__restrict__ w, long long n, unsigned k0, unsigned k1) {
    const long long nblk = (n + 3) / 4;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < nblk;
         g += (long long)gridDim.x * blockDim.x) {
        const uint4 x = philox4x32_10((unsigned)g, (unsigned)(g >> 32), k0, k1);
        float z[4];
        const float r01 = sqrtf(-2.0f * logf(unit_uniform(x.x)));
        const float r23 = sqrtf(-2.0f * logf(unit_uniform(x.z)));
        float s1, c1, s3, c3;
        sincospif(2.0f * unit_uniform(x.y), &s1, &c1);
        sincospif(2.0f * unit_uniform(x.w), &s3, &c3);
        z[0] = r01 * c1;
        z[1] = r01 * s1;
        z[2] = r23 * c3;
        z[3] = r23 * s3;
        const long long i0 = 4 * g;
        if (i0 + 4 <= n && (reinterpret_cast<uintptr_t>(w) & 15) == 0) {
            *reinterpret_cast<float4 *>(w + i0) = make_float4(z[0], z[1], z[2], z[3]);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (i0 + e < n) w[i0 + e] = z[e];
        }
    }
}

__global__ void k_colour(cufftComplex *ck, int N, const float *__restrict__ amp) {
    const int Nz = N / 2 + 1;
    const long long n = (long long)N * N * Nz;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int kz = (int)(idx % Nz);
        const long long t = idx / Nz;
        const int ky = (int)(t % N);
        const int kx = (int)(t / N);
        const int nx = wavenumber(kx, N), ny = wavenumber(ky, N);
        const float a = amp[nx * nx + ny * ny + kz * kz];
        cufftComplex v = ck[idx];
        v.x *= a;
        v.y *= a;
        ck[idx] = v;
    }
}

// Adjoint of colouring after the inverse Laplacian: out = in * amp(k) / Lambda(k), k = 0 -> 0;
// Lambda the FDA-2 symbol from s_half, or (lap1 not null) the order-n symbol sum of lap1.
__global__ void k_adj_colour(const cufftComplex *in, cufftComplex *out, int N, const float *__restrict__ amp,
                             const float *s_half, float inv_d2, const float *__restrict__ lap1) {
    const int Nz = N / 2 + 1;
    const long long n = (long long)N * N * Nz;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int kz = (int)(idx % Nz);
        const long long t = idx / Nz;
        const int ky = (int)(t % N);
        const int kx = (int)(t / N);
        const int nx = wavenumber(kx, N), ny = wavenumber(ky, N);
        const int n2 = nx * nx + ny * ny + kz * kz;
        float m = 0.0f;
        if (n2 > 0) {
            const float sx = s_half[kx], sy = s_half[ky], sz = s_half[kz];
            const float lam = lap1 ? lap1[kx] + lap1[ky] + lap1[kz] : -4.0f * inv_d2 * (sx * sx + sy * sy + sz * sz);
            m = amp[n2] / lam;
        }
        cufftComplex v = in[idx];
        v.x *= m;
        v.y *= m;
        out[idx] = v;
    }
}

__global__ void k_inv_lap(const cufftComplex *in, cufftComplex *out, int N, const float *s_half,
                          float inv_d2, float scale) {
    const int Nz = N / 2 + 1;
    const long long n = (long long)N * N * Nz;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int kz = (int)(idx % Nz);
        const long long t = idx / Nz;
        const int ky = (int)(t % N);
        const int kx = (int)(t / N);
        const float sx = s_half[kx], sy = s_half[ky], sz = s_half[kz];
        const float lam = -4.0f * inv_d2 * (sx * sx + sy * sy + sz * sz);
        cufftComplex v = in[idx];
        const float m = (lam != 0.0f) ? scale / lam : 0.0f;
        v.x *= m;
        v.y *= m;
        out[idx] = v;
    }
}

// Order-4/6 inverse Laplacian: Lambda(k) = sum over axes of the 1D second-derivative symbol
// (lap1, per grid index, including 1/d^2).
__global__ void k_inv_lap_sym(const cufftComplex *in, cufftComplex *out, int N, const float *lap1, float scale) {
    const int Nz = N / 2 + 1;
    const long long n = (long long)N * N * Nz;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int kz = (int)(idx % Nz);
        const long long t = idx / Nz;
        const int ky = (int)(t % N);
        const int kx = (int)(t / N);
        const float lam = lap1[kx] + lap1[ky] + lap1[kz];
        cufftComplex v = in[idx];
        const float m = (lam != 0.0f) ? scale / lam : 0.0f;
        v.x *= m;
        v.y *= m;
        out[idx] = v;
    }
}

// Periodic central gradient of FDA order ORDER at the LPT grid nodes.
template <int ORDER>
__global__ void k_gradient_n(const float *phi, float *psi, int N, float inv_d) {
    const long long N3 = (long long)N * N * N;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N3;
         idx += (long long)gridDim.x * blockDim.x) {
        const int c[3] = {(int)(idx / ((long long)N * N)), (int)((idx / N) % N), (int)(idx % N)};
        const long long st[3] = {(long long)N * N, N, 1};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float g = 0.0f;
#pragma unroll
            for (int m = 1; m <= Fda<ORDER>::ng; ++m) {
                const int p = c[a] + m >= N ? c[a] + m - N : c[a] + m;
                const int q = c[a] - m < 0 ? c[a] - m + N : c[a] - m;
                g = fmaf(Fda<ORDER>::g(m), phi[idx + (p - c[a]) * st[a]] - phi[idx + (q - c[a]) * st[a]], g);
            }
            psi[a * N3 + idx] = g * inv_d;
        }
    }
}

__global__ void k_second_derivative(const cufftComplex *in, cufftComplex *out, int N,
                                    const float *s_full, int ai, int aj) {
    const int Nz = N / 2 + 1;
    const long long n = (long long)N * N * Nz;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        int c[3];
        c[2] = (int)(idx % Nz);
        const long long t = idx / Nz;
        c[1] = (int)(t % N);
        c[0] = (int)(t / N);
        const float m = -s_full[c[ai]] * s_full[c[aj]];
        cufftComplex v = in[idx];
        v.x *= m;
        v.y *= m;
        out[idx] = v;
    }
}

__global__ void k_source_init(const float *xx, const float *yy, const float *zz, float *S,
                              long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float a = xx[i], b = yy[i], c = zz[i];
        S[i] = a * b + a * c + b * c;
    }
}

__global__ void k_source_sub(const float *t, float *S, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float v = t[i];
        S[i] -= v * v;
    }
}

__global__ void k_gradient(const float *phi, float *psi, int N, float inv_2d) {
    const long long N3 = (long long)N * N * N;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N3;
         idx += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(idx % N);
        const long long t = idx / N;
        const int j = (int)(t % N);
        const int i = (int)(t / N);
        const long long NN = (long long)N * N;
        const int ip = i + 1 == N ? 0 : i + 1, im = i == 0 ? N - 1 : i - 1;
        const int jp = j + 1 == N ? 0 : j + 1, jm = j == 0 ? N - 1 : j - 1;
        const int kp = k + 1 == N ? 0 : k + 1, km = k == 0 ? N - 1 : k - 1;
        const long long row = (long long)i * NN + (long long)j * N;
        psi[idx] = (phi[(long long)ip * NN + (long long)j * N + k] -
                    phi[(long long)im * NN + (long long)j * N + k]) * inv_2d;
        psi[N3 + idx] = (phi[(long long)i * NN + (long long)jp * N + k] -
                         phi[(long long)i * NN + (long long)jm * N + k]) * inv_2d;
        psi[2 * N3 + idx] = (phi[row + kp] - phi[row + km]) * inv_2d;
    }
}

int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    return (int)(g < 8192 ? (g > 0 ? g : 1) : 8192);
}

}  // namespace

cudaError_t launch_white_noise(Ctx &c, unsigned long long seed, float *w) {
    const long long nblk = (c.N3 + 3) / 4;
    long long grid = (nblk + 255) / 256;
    if (grid > 8 * (long long)c.num_sms * 8) grid = 8 * (long long)c.num_sms * 8;
    if (grid < 1) grid = 1;
    k_white_noise<<<(int)grid, 256, 0, c.stream>>>(w, c.N3, (unsigned)seed, (unsigned)(seed >> 32));
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_colour(Ctx &c, cufftComplex *ck) {
    const int N = c.Np;
    const long long n = (long long)N * N * (N / 2 + 1);
    k_colour<<<grid_for(n, 256), 256, 0, c.stream>>>(ck, N, c.table_arena + c.amp_off);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_adj_colour(Ctx &c, const cufftComplex *in, cufftComplex *out) {
    const int N = c.Np;
    const long long n = (long long)N * N * (N / 2 + 1);
    const double d = c.L / N;
    k_adj_colour<<<grid_for(n, 256), 256, 0, c.stream>>>(
        in, out, N, c.table_arena + c.amp_off, c.table_arena + c.sin_half_off, (float)(1.0 / (d * d)),
        c.prm.fda_order != 2 ? c.table_arena + c.lap1_off : nullptr);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_inv_laplacian(Ctx &c, const cufftComplex *in, cufftComplex *out, float scale) {
    const int N = c.Np;
    const long long n = (long long)N * N * (N / 2 + 1);
    const double d = c.L / N;
    if (c.prm.fda_order != 2)
        k_inv_lap_sym<<<grid_for(n, 256), 256, 0, c.stream>>>(in, out, N, c.table_arena + c.lap1_off, scale);
    else
        k_inv_lap<<<grid_for(n, 256), 256, 0, c.stream>>>(in, out, N, c.table_arena + c.sin_half_off,
                                                           (float)(1.0 / (d * d)), scale);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_second_derivative(Ctx &c, const cufftComplex *in, cufftComplex *out, int i,
                                     int j) {
    const int N = c.Np;
    const long long n = (long long)N * N * (N / 2 + 1);
    k_second_derivative<<<grid_for(n, 256), 256, 0, c.stream>>>(
        in, out, N, c.table_arena + (c.prm.fda_order != 2 ? c.grad1_off : c.sin_full_off), i, j);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_source_init(Ctx &c, const float *xx, const float *yy, const float *zz,
                               float *S) {
    k_source_init<<<grid_for(c.N3, 256), 256, 0, c.stream>>>(xx, yy, zz, S, c.N3);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_source_sub(Ctx &c, const float *t, float *S) {
    k_source_sub<<<grid_for(c.N3, 256), 256, 0, c.stream>>>(t, S, c.N3);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_gradient(Ctx &c, const float *phi, float *psi) {
    const double d = c.L / c.Np;
    switch (c.prm.fda_order) {
        case 4: k_gradient_n<4><<<grid_for(c.N3, 256), 256, 0, c.stream>>>(phi, psi, c.Np, (float)(1.0 / d)); break;
        case 6: k_gradient_n<6><<<grid_for(c.N3, 256), 256, 0, c.stream>>>(phi, psi, c.Np, (float)(1.0 / d)); break;
        default: k_gradient<<<grid_for(c.N3, 256), 256, 0, c.stream>>>(phi, psi, c.Np, (float)(0.5 / d));
    }
    ++c.launches;
    return cudaGetLastError();
}

}  // namespace scola
