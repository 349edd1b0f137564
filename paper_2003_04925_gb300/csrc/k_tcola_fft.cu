// Periodic Poisson solve of the full-box tCOLA forces (Sec. 2.2 with the FDA-2 Laplacian):
// Phi = IDFT[ DFT[delta] / (lap(kx) + lap(ky) + lap(kz)) ] / N^3 on the N^3 grid, k = 0 removed,
// with the shared-memory FFTs of fft_util.cuh in five mesh passes.  Each pass reads rows
// whose transform axis is contiguous and writes them so that the next pass again finds its
// axis contiguous:
//   1 x forward, real -> half spectrum:  delta[z][y][x]   -> A[kx][z][y]   (kx <= N/2)
//   2 y forward:                          A[kx][z][y]      -> B[ky][kx][z]
//   3 z forward, Green's function, z inverse:
//                                         B[ky][kx][kz]    -> A[z][kx][ky]
//   4 y inverse:                          A[z][kx][ky]     -> B[y][z][kx]
//   5 x inverse, half spectrum -> real:   B[y][z][kx]      -> Phi[z][y][x]
// Two real rows share one complex transform in passes 1 and 5 (z = x' + i x'': X'_k =
// (Z_k + conj Z_{N-k}) / 2, X''_k = (Z_k - conj Z_{N-k}) / (2 i); backwards the two Hermitian
// half spectra are extended and combined as X' + i X'').  A power-of-two N is transformed
// directly; any other N by Bluestein's chirp convolution of a power-of-two length L >= 2N - 1
// (w_n = exp(i pi n^2 / N), spectrum of the chirp kernel tabulated on the host in FP64; the
// inverse DFT as the conjugate of the forward DFT of the conjugate).  FP32 throughout.
//
// A CTA serves tiles of R rows in turn.  Where every tile's rows start and end 16-byte
// aligned, the rows of the next tile are fetched into a staging buffer by bulk asynchronous
// copies (one mbarrier, bounded waits) as soon as the current tile's first FFT stage has read
// its own; otherwise the first stage loads from global memory directly.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "device_util.cuh"
#include "fft_util.cuh"
#include "tc_util.cuh"

namespace scola {

namespace {

constexpr int kFtThreads = 256;
constexpr int kFtSpan = 2048;                    // complex values per transform batch (R rows x L)
constexpr int kFtMaxRows = 256;                  // R cap (tiny grids)
constexpr int kFtStage = 20480;                  // staging bytes: the largest tile input (R <= 256)

enum FtPass { FT_X_FWD = 1, FT_Y_FWD = 2, FT_Z_SOLVE = 3, FT_Y_INV = 4, FT_X_INV = 5 };

struct FtArgs {
    int N, NX, L, logL, R, blue, ntiles;
    int *err;                 // bit 1 set if a staged copy's bounded wait expired
    float invL, inv_n3;
    const float2 *tw;         // exp(-2 pi i e / L), e < L
    const float2 *w256;       // the radix-16 second-stage twiddles
    const float2 *w;          // Bluestein chirp w_n, n < N
    const float2 *Bk;         // Bluestein: DFT_L of the chirp kernel
    const float *lap;         // 1D FDA-2 symbol per index, N
    const float *in_r;        // pass 1 input (real)
    const float2 *in_c;       // passes 2-5 input
    float2 *out_c;            // passes 1-4 output
    float *out_r;             // pass 5 output (real)
};

using fft::cmul;
using fft::cmulc;

// Shared-memory geometry of one pass's row transforms.
struct Rows {
    int N, L, logL, R, Ls, blue;
    float invL;
    const float2 *tw, *w, *Bk, *w256;
};

// DFT of R rows of length N (SIGN -1 forward, +1 inverse, unnormalised), x_n = load(r, n);
// load may read `spare`, never `dst`.  Returns the buffer to read with row_get.
template <int SIGN, class Load, class Hook = fft::NoHook>
__device__ float2 *row_dft(const Rows &F, Load load, float2 *dst, float2 *spare, Hook after_first = Hook()) {
    if (!F.blue) return fft::transform<SIGN>(load, dst, spare, F.R, F.logL, F.tw, F.w256, after_first);
    const float2 *w = F.w;
    const int N = F.N;
    auto chirped = [&](int r, int n) {
        if (n >= N) return make_float2(0.f, 0.f);
        float2 x = load(r, n);
        if (SIGN > 0) x.y = -x.y;
        return cmulc(x, w[n]);
    };
    float2 *f = fft::transform<-1>(chirped, dst, spare, F.R, F.logL, F.tw, F.w256, after_first);
    float2 *g = f == dst ? spare : dst;
    const float2 *fc = f, *Bk = F.Bk;
    const int Ls = F.Ls;
    auto product = [&](int r, int n) { return cmul(fc[r * Ls + fft::pad(n)], Bk[n]); };
    return fft::transform<+1>(product, g, f, F.R, F.logL, F.tw, F.w256);
}

// Element k of row r of the DFT that row_dft left in res.
template <int SIGN>
__device__ __forceinline__ float2 row_get(const Rows &F, const float2 *res, int r, int k) {
    const float2 v = res[r * F.Ls + fft::pad(k)];
    if (!F.blue) return v;
    float2 X = cmulc(v, F.w[k]);
    X.x *= F.invL;
    X.y *= F.invL;
    if (SIGN > 0) X.y = -X.y;
    return X;
}

// rows per tile and the complex values of one shared-memory buffer of them
int ft_rows(int L) { return std::min(kFtSpan / L, kFtMaxRows); }
int ft_buf(int L) { return ft_rows(L) * fft::row_stride(L, ft_rows(L)); }

size_t ft_smem_bytes(int N, int L) {
    return 16 + kFtStage + sizeof(float2) * ((size_t)2 * ft_buf(L) + fft::kW256 + 2 * L + N) + sizeof(float) * N;
}

// Issue (warp 0) the bulk copies of tile t's input rows into st; their byte count arrives on bar.
template <int PASS>
__device__ void issue_tile(const FtArgs &A, int t, unsigned char *st, uint64_t *bar) {
    const int N = A.N, NX = A.NX, R = A.R, lane = threadIdx.x & 31;
    const long long N2 = (long long)N * N;
    const char *src = nullptr;
    uint32_t bytes = 0;
    if (PASS == FT_X_FWD) {
        const long long rr0 = (long long)t * 2 * R;
        src = reinterpret_cast<const char *>(A.in_r + rr0 * N);
        bytes = (uint32_t)(min((long long)2 * R, N2 - rr0) * N * 4);
    } else if (PASS == FT_X_INV) {
        const long long rr0 = (long long)t * 2 * R;
        src = reinterpret_cast<const char *>(A.in_c + rr0 * NX);
        bytes = (uint32_t)(min((long long)2 * R, N2 - rr0) * NX * 8);
    } else if (PASS == FT_Y_FWD || PASS == FT_Y_INV) {
        const long long nrows = (long long)N * NX, r0 = (long long)t * R;
        src = reinterpret_cast<const char *>(A.in_c + r0 * N);
        bytes = (uint32_t)(min((long long)R, nrows - r0) * N * 8);
    }
    if (PASS != FT_Z_SOLVE) {
        if (lane == 0) {
            tc::mbar_arrive_expect_tx(bar, bytes);
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    tc::smem_u32(st)),
                "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
                : "memory");
        }
        return;
    }
    // z solve: R rows (ky0 + r, kx), each N complex values, to st + r N
    const int kx = t % NX, ky0 = (t / NX) * R, nr = min(R, N - ky0);
    if (lane == 0) tc::mbar_arrive_expect_tx(bar, (uint32_t)(nr * N * 8));
    __syncwarp();
    for (int r = lane; r < nr; r += 32) {
        const float2 *row = A.in_c + ((long long)(ky0 + r) * NX + kx) * N;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                tc::smem_u32(st + (size_t)r * N * 8)),
            "l"(row), "r"((uint32_t)(N * 8)), "r"(tc::smem_u32(bar))
            : "memory");
    }
}

template <int PASS, bool BULK>
__global__ void __launch_bounds__(kFtThreads, 2) k_tc_fft(const FtArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = A.N, NX = A.NX, L = A.L, R = A.R;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    unsigned char *st = smem + 16;
    const float *stf = reinterpret_cast<const float *>(st);
    const float2 *stc = reinterpret_cast<const float2 *>(st);
    const int Ls = fft::row_stride(L, R);
    float2 *b0 = reinterpret_cast<float2 *>(st + kFtStage);
    float2 *b1 = b0 + R * Ls;
    float2 *w256 = b1 + R * Ls;      // 256
    float2 *tw = w256 + fft::kW256;  // L
    float2 *Bk = tw + L;             // L (Bluestein)
    float2 *w = Bk + L;              // N (Bluestein)
    float *lap = reinterpret_cast<float *>(w + N);
    for (int q = threadIdx.x; q < fft::kW256; q += kFtThreads) w256[q] = A.w256[q];
    for (int q = threadIdx.x; q < L; q += kFtThreads) {
        tw[q] = A.tw[q];
        if (A.blue) Bk[q] = A.Bk[q];
    }
    for (int q = threadIdx.x; q < N; q += kFtThreads) {
        if (A.blue) w[q] = A.w[q];
        lap[q] = A.lap[q];
    }
    __syncthreads();
    Rows F;
    F.N = N;
    F.L = L;
    F.logL = A.logL;
    F.R = R;
    F.Ls = Ls;
    F.blue = A.blue;
    F.invL = A.invL;
    F.tw = tw;
    F.w = w;
    F.Bk = Bk;
    F.w256 = w256;
    const int N2 = N * N, logR = __ffs(R) - 1;
    if (BULK) {
        if (threadIdx.x == 0) {
            tc::mbar_init(bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (threadIdx.x < 32 && (int)blockIdx.x < A.ntiles) issue_tile<PASS>(A, blockIdx.x, st, bar);
    }
    uint32_t parity = 0;
    // after the first stage of a tile has read the staging buffer: fetch the next tile's rows
    auto prefetch = [&](int t) {
        if (!BULK) return;
        if (threadIdx.x < 32 && t + (int)gridDim.x < A.ntiles) {
            tc::fence_proxy_async();
            issue_tile<PASS>(A, t + gridDim.x, st, bar);
        }
    };
    for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
        if (BULK) {
            volatile int no_abort = 0;
            if (!tc::mbar_wait(bar, parity, &no_abort)) {
                if (threadIdx.x == 0) atomicOr(A.err, 1);
                tc::mbar_wait(bar, parity, &no_abort);       // the copy in flight, once more, bounded
                return;
            }
            parity ^= 1u;
        }
        auto hook = [&]() { prefetch(t); };
        // (indices fit 32 bits: N <= 1024, so N^2 (N / 2 + 1) < 2^30)
        if (PASS == FT_X_FWD) {
            // real rows (z, y) = rr0 + 2 r + s, s = 0, 1
            const int rr0 = t * 2 * R;
            const float *in = A.in_r;
            auto load = [&](int r, int n) {
                const int a = rr0 + 2 * r;
                if (BULK)
                    return make_float2(a < N2 ? stf[2 * r * N + n] : 0.f, a + 1 < N2 ? stf[(2 * r + 1) * N + n] : 0.f);
                return make_float2(a < N2 ? in[a * N + n] : 0.f, a + 1 < N2 ? in[(a + 1) * N + n] : 0.f);
            };
            const float2 *res = row_dft<-1>(F, load, b0, b1, hook);
            for (int q = threadIdx.x; q < (NX << (logR + 1)); q += kFtThreads) {
                const int kx = q >> (logR + 1), i = q & (2 * R - 1);
                const int rr = rr0 + i;
                if (rr >= N2) continue;
                const int r = i >> 1;
                const float2 Zk = row_get<-1>(F, res, r, kx), Zm = row_get<-1>(F, res, r, kx == 0 ? 0 : N - kx);
                const float2 X = (i & 1) ? make_float2(0.5f * (Zk.y + Zm.y), -0.5f * (Zk.x - Zm.x))
                                         : make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y));
                A.out_c[kx * N2 + rr] = X;
            }
        } else if (PASS == FT_Y_FWD || PASS == FT_Y_INV) {
            // rows (kx, z) [forward] or (z, kx) [inverse], row index rho < N NX
            const int nrows = N * NX;
            const int r0 = t * R;
            const float2 *in = A.in_c;
            auto load = [&](int r, int n) {
                const int rho = r0 + r;
                if (rho >= nrows) return make_float2(0.f, 0.f);
                return BULK ? stc[r * N + n] : in[rho * N + n];
            };
            const float2 *res =
                PASS == FT_Y_FWD ? row_dft<-1>(F, load, b0, b1, hook) : row_dft<+1>(F, load, b0, b1, hook);
            for (int q = threadIdx.x; q < (N << logR); q += kFtThreads) {
                const int k = q >> logR, r = q & (R - 1);
                const int rho = r0 + r;
                if (rho >= nrows) continue;
                const float2 v = PASS == FT_Y_FWD ? row_get<-1>(F, res, r, k) : row_get<+1>(F, res, r, k);
                A.out_c[k * nrows + rho] = v;
            }
        } else if (PASS == FT_Z_SOLVE) {
            // rows (ky, kx): tile = R consecutive ky at one kx
            const int kx = t % NX, ky0 = (t / NX) * R;
            const float2 *in = A.in_c;
            auto load = [&](int r, int n) {
                const int ky = ky0 + r;
                if (ky >= N) return make_float2(0.f, 0.f);
                return BULK ? stc[r * N + n] : in[(ky * NX + kx) * N + n];
            };
            const float2 *res = row_dft<-1>(F, load, b0, b1, hook);
            float2 *spare = const_cast<float2 *>(res);
            float2 *dst = res == b0 ? b1 : b0;
            const float inv_n3 = A.inv_n3;
            const float lx = lap[kx];
            auto green = [&](int r, int kz) {
                const int ky = ky0 + r;
                const float2 v = row_get<-1>(F, res, r, kz);
                if (ky >= N || (kx == 0 && ky == 0 && kz == 0)) return make_float2(0.f, 0.f);
                // (the symbol sum is at most 12 / dg^2 in magnitude, far inside __fdividef's range)
                const float g = __fdividef(inv_n3, lx + lap[ky] + lap[kz]);
                return make_float2(v.x * g, v.y * g);
            };
            const float2 *out = row_dft<+1>(F, green, dst, spare);
            for (int q = threadIdx.x; q < (N << logR); q += kFtThreads) {
                const int z = q >> logR, r = q & (R - 1);
                const int ky = ky0 + r;
                if (ky >= N) continue;
                A.out_c[(z * NX + kx) * N + ky] = row_get<+1>(F, out, r, z);
            }
        } else {   // FT_X_INV: half-spectrum rows (y, z) = rr0 + 2 r + s
            const int rr0 = t * 2 * R;
            const float2 *in = A.in_c;
            const int half = N / 2;
            const bool even = (N & 1) == 0;
            auto herm = [&](int a, int n) {                 // X_n of half row a, Hermitian-extended
                if (a >= N2) return make_float2(0.f, 0.f);
                const float2 *row = BULK ? stc + (a - rr0) * NX : in + a * NX;
                if (n <= half) {
                    float2 v = row[n];
                    if (n == 0 || (even && n == half)) v.y = 0.f;
                    return v;
                }
                const float2 v = row[N - n];
                return make_float2(v.x, -v.y);
            };
            auto load = [&](int r, int n) {
                const int a = rr0 + 2 * r;
                const float2 X1 = herm(a, n), X2 = herm(a + 1, n);
                return make_float2(X1.x - X2.y, X1.y + X2.x);
            };
            const float2 *res = row_dft<+1>(F, load, b0, b1, hook);
            // one warp per output row (y, z), lanes along x
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            for (int i = warp; i < 2 * R; i += kFtThreads / 32) {
                const int rr = rr0 + i;                     // = y N + z
                if (rr >= N2) break;
                const int y = rr / N, z = rr - y * N;
                float *dst = A.out_r + (z * N + y) * N;
                for (int x = lane; x < N; x += 32) {
                    const float2 v = row_get<+1>(F, res, i >> 1, x);
                    dst[x] = (i & 1) ? v.y : v.x;
                }
            }
        }
        __syncthreads();
    }
}

template <int PASS>
cudaError_t set_ft_attr() {
    const int bytes = (int)ft_smem_bytes(1024, 2048);
    cudaError_t e = cudaFuncSetAttribute(k_tc_fft<PASS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_tc_fft<PASS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// Whether every tile of the pass has 16-byte aligned input rows (start and length) that fit
// the staging buffer: the condition of the bulk copies.
template <int PASS>
bool ft_bulk_ok(const FtArgs &a) {
    const long long N = a.N, NX = a.NX, R = a.R, N2 = N * N;
    const void *base = PASS == FT_X_FWD ? (const void *)a.in_r : (const void *)a.in_c;
    if (reinterpret_cast<uintptr_t>(base) % 16) return false;
    long long row_bytes, tile_rows, rows;
    switch (PASS) {
        case FT_X_FWD: row_bytes = 4 * N; tile_rows = 2 * R; rows = N2; break;
        case FT_X_INV: row_bytes = 8 * NX; tile_rows = 2 * R; rows = N2; break;
        case FT_Z_SOLVE: return (8 * N) % 16 == 0 && R * 8 * N <= kFtStage;
        default: row_bytes = 8 * N; tile_rows = R; rows = N * NX;
    }
    return (tile_rows * row_bytes) % 16 == 0 && ((rows % tile_rows) * row_bytes) % 16 == 0 &&
           tile_rows * row_bytes <= kFtStage;
}

template <int PASS>
cudaError_t run_ft_pass(Ctx &c, FtArgs a) {
    const int N = a.N, R = a.R;
    switch (PASS) {
        case FT_X_FWD:
        case FT_X_INV: a.ntiles = (int)(((long long)N * N + 2 * R - 1) / (2 * R)); break;
        case FT_Z_SOLVE: a.ntiles = a.NX * ((N + R - 1) / R); break;
        default: a.ntiles = (int)(((long long)N * a.NX + R - 1) / R);
    }
    const size_t smem = ft_smem_bytes(N, a.L);
    const bool bulk = ft_bulk_ok<PASS>(a);
    int per_sm = 1;
    const cudaError_t oe =
        bulk ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tc_fft<PASS, true>, kFtThreads, smem)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tc_fft<PASS, false>, kFtThreads, smem);
    if (oe != cudaSuccess || per_sm < 1) per_sm = 1;
    const int grid = std::max(1, std::min(a.ntiles, c.num_sms * per_sm));
    if (bulk) k_tc_fft<PASS, true><<<grid, kFtThreads, smem, c.stream>>>(a);
    else k_tc_fft<PASS, false><<<grid, kFtThreads, smem, c.stream>>>(a);
    ++c.launches;
    return cudaGetLastError();
}

}  // namespace

void tc_fft_plan(int N, int &L, int &logL, int &R, bool &blue) {
    blue = (N & (N - 1)) != 0;
    const int need = blue ? 2 * N - 1 : N;
    L = 2;
    logL = 1;
    while (L < need) {
        L <<= 1;
        ++logL;
    }
    R = ft_rows(L);
}

bool tc_fft_supported(int N) {
    if (N < 2) return false;
    int L, logL, R;
    bool blue;
    tc_fft_plan(N, L, logL, R, blue);
    return R >= 1 && L <= kFtSpan && ft_smem_bytes(N, L) <= ft_smem_bytes(1024, 2048);
}

void tc_fft_tables(int N, std::vector<float> &arena, long long &tw_off, long long &w_off, long long &bk_off) {
    int L, logL, R;
    bool blue;
    tc_fft_plan(N, L, logL, R, blue);
    auto even = [&]() {
        if (arena.size() & 1) arena.push_back(0.0f);
        return (long long)arena.size();
    };
    std::vector<double> cs(L), sn(L);
    for (int j = 0; j < L; ++j) {
        cs[j] = std::cos(2.0 * M_PI * j / L);
        sn[j] = std::sin(2.0 * M_PI * j / L);
    }
    tw_off = even();
    for (int j = 0; j < L; ++j) {
        arena.push_back((float)cs[j]);
        arena.push_back((float)-sn[j]);
    }
    w_off = bk_off = tw_off;
    if (!blue) return;
    // chirp w_n = exp(i pi n^2 / N) (phase reduced exactly: n^2 mod 2N) and the DFT_L of the
    // kernel b_m = w_|m|, |m| < N (wrapped), a direct FP64 sum
    std::vector<double> wr(N), wi(N);
    for (int n = 0; n < N; ++n) {
        const long long e = ((long long)n * n) % (2LL * N);
        wr[n] = std::cos(M_PI * (double)e / N);
        wi[n] = std::sin(M_PI * (double)e / N);
    }
    w_off = even();
    for (int n = 0; n < N; ++n) {
        arena.push_back((float)wr[n]);
        arena.push_back((float)wi[n]);
    }
    std::vector<double> br(L, 0.0), bi(L, 0.0);
    for (int m = 0; m < N; ++m) {
        br[m] = wr[m];
        bi[m] = wi[m];
        if (m > 0) {
            br[L - m] = wr[m];
            bi[L - m] = wi[m];
        }
    }
    bk_off = even();
    for (int k = 0; k < L; ++k) {
        double re = 0.0, im = 0.0;
        for (int m = 0; m < L; ++m) {
            if (br[m] == 0.0 && bi[m] == 0.0) continue;
            const int j = (int)(((long long)k * m) % L);
            re += br[m] * cs[j] + bi[m] * sn[j];
            im += bi[m] * cs[j] - br[m] * sn[j];
        }
        arena.push_back((float)re);
        arena.push_back((float)im);
    }
}

cudaError_t init_tc_fft_kernels() {
    cudaError_t e;
    if ((e = set_ft_attr<FT_X_FWD>())) return e;
    if ((e = set_ft_attr<FT_Y_FWD>())) return e;
    if ((e = set_ft_attr<FT_Z_SOLVE>())) return e;
    if ((e = set_ft_attr<FT_Y_INV>())) return e;
    return set_ft_attr<FT_X_INV>();
}

cudaError_t launch_tc_poisson(Ctx &c, const float *delta, float *phi) {
    FtArgs a;
    const int N = c.tc_ng;
    bool blue;
    tc_fft_plan(N, a.L, a.logL, a.R, blue);
    a.N = N;
    a.NX = N / 2 + 1;
    a.blue = blue ? 1 : 0;
    a.ntiles = 0;
    a.err = c.dev_err;
    a.invL = 1.0f / (float)a.L;
    a.inv_n3 = (float)(1.0 / (double)c.tc_n3);
    a.tw = reinterpret_cast<const float2 *>(c.table_arena + c.tc_fft_tw_off);
    a.w256 = reinterpret_cast<const float2 *>(c.table_arena + c.fft_w256_off);
    a.w = reinterpret_cast<const float2 *>(c.table_arena + c.tc_fft_w_off);
    a.Bk = reinterpret_cast<const float2 *>(c.table_arena + c.tc_fft_bk_off);
    a.lap = c.table_arena + c.tc_lap_off;
    float2 *A1 = reinterpret_cast<float2 *>(c.tc_dk), *B1 = reinterpret_cast<float2 *>(c.tc_dk2);
    cudaError_t e;
    a.in_r = delta;
    a.in_c = nullptr;
    a.out_c = A1;
    a.out_r = nullptr;
    if ((e = run_ft_pass<FT_X_FWD>(c, a))) return e;
    a.in_c = A1;
    a.out_c = B1;
    if ((e = run_ft_pass<FT_Y_FWD>(c, a))) return e;
    a.in_c = B1;
    a.out_c = A1;
    if ((e = run_ft_pass<FT_Z_SOLVE>(c, a))) return e;
    a.in_c = A1;
    a.out_c = B1;
    if ((e = run_ft_pass<FT_Y_INV>(c, a))) return e;
    a.in_c = B1;
    a.out_c = nullptr;
    a.out_r = phi;
    return run_ft_pass<FT_X_INV>(c, a);
}

}  // namespace scola
