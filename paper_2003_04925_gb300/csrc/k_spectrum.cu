// Binned power spectrum of a density field on the N^3 LPT grid (Sec. 4.2, Eq. 24 with
// the normalisation P = L^3 <|DFT delta|^2> / N^6).
//
// The field is transformed with cuFFT (R2C, unnormalised).  The half spectrum holds every
// mode of the full spectrum once (planes kz = 0 and kz = N/2) or twice (0 < kz < N/2, the
// conjugate partner having the same |k| and |delta_k|^2), so each half-spectrum mode enters
// its bin with that weight.  The bin of a mode depends only on the integer n^2 = nx^2 +
// ny^2 + nz^2 of its wrapped wavenumbers: the host assigns bins per n^2 in FP64 and the
// kernel looks them up.  Sums are FP64; every CTA reduces its modes into its own row of
// partial sums, and a second kernel adds the rows in a fixed order (deterministic).
#include "device_util.cuh"

namespace scola {

namespace {

constexpr int kSpecThreads = 256;

// Per CTA and bin: weighted sum of |delta_k|^2, of sqrt(n^2), and the mode count.
__global__ void __launch_bounds__(kSpecThreads)
k_spectrum_partial(const cufftComplex *__restrict__ dk, int N, const int *__restrict__ bin_of_n2, int nbins,
                   double *__restrict__ part_p, double *__restrict__ part_k, unsigned long long *__restrict__ part_n) {
    extern __shared__ unsigned char sm[];
    double *sp = reinterpret_cast<double *>(sm);
    double *sk = sp + nbins;
    unsigned long long *sn = reinterpret_cast<unsigned long long *>(sk + nbins);
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        sp[b] = 0.0;
        sk[b] = 0.0;
        sn[b] = 0ull;
    }
    __syncthreads();
    const int Nz = N / 2 + 1;
    const long long n = (long long)N * N * Nz;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int kz = (int)(idx % Nz);
        const long long t = idx / Nz;
        const int ky = (int)(t % N), kx = (int)(t / N);
        const int nx = kx <= N / 2 ? kx : kx - N, ny = ky <= N / 2 ? ky : ky - N;
        const int n2 = nx * nx + ny * ny + kz * kz;
        const int b = bin_of_n2[n2];
        if (b < 0) continue;
        const unsigned w = (kz == 0 || 2 * kz == N) ? 1u : 2u;
        const cufftComplex v = dk[idx];
        const double p = (double)v.x * v.x + (double)v.y * v.y;
        atomicAdd(&sp[b], w * p);
        atomicAdd(&sk[b], w * sqrt((double)n2));
        atomicAdd(&sn[b], (unsigned long long)w);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        part_p[(long long)blockIdx.x * nbins + b] = sp[b];
        part_k[(long long)blockIdx.x * nbins + b] = sk[b];
        part_n[(long long)blockIdx.x * nbins + b] = sn[b];
    }
}

// Adds the CTAs' rows in order of CTA index (one thread per bin).
__global__ void k_spectrum_sum(const double *__restrict__ part_p, const double *__restrict__ part_k,
                               const unsigned long long *__restrict__ part_n, int rows, int nbins,
                               double *__restrict__ out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    double p = 0.0, k = 0.0;
    unsigned long long c = 0;
    for (int r = 0; r < rows; ++r) {
        p += part_p[(long long)r * nbins + b];
        k += part_k[(long long)r * nbins + b];
        c += part_n[(long long)r * nbins + b];
    }
    out[b] = p;
    out[nbins + b] = k;
    out[2 * nbins + b] = (double)c;
}

}  // namespace

cudaError_t launch_spectrum(Ctx &c, const cufftComplex *dk, const int *bin_of_n2, int nbins, double *scratch,
                            int rows, double *out) {
    double *part_p = scratch, *part_k = scratch + (long long)rows * nbins;
    unsigned long long *part_n = reinterpret_cast<unsigned long long *>(scratch + 2LL * rows * nbins);
    const size_t smem = (size_t)nbins * (2 * sizeof(double) + sizeof(unsigned long long));
    k_spectrum_partial<<<rows, kSpecThreads, smem, c.stream>>>(dk, c.Np, bin_of_n2, nbins, part_p, part_k, part_n);
    ++c.launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_spectrum_sum<<<(nbins + 127) / 128, 128, 0, c.stream>>>(part_p, part_k, part_n, rows, nbins, out);
    ++c.launches;
    return cudaGetLastError();
}

}  // namespace scola
