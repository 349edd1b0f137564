// Dirichlet Poisson solve with fast sine transforms on the CUDA cores: O(Ng log Ng) per
// pencil, pencils held in shared memory (App. C, Eqs. 63-71).
//
// DST-I of length N, S_j = sum_{n=1..N} x_n sin(pi j n / P), P = N + 1, from one real DFT of
// length P.  With x_0 = x_P = 0 and theta = pi / P form
//   y_n = sin(n theta) (x_n + x_{P-n}) + (x_n - x_{P-n}) / 2,   n = 0 .. P-1.
// Its DFT Y_k = R_k - i I_k (R: cosine sums, I: sine sums) gives
//   S_{2k} = I_k,   S_1 = R_0 / 2,   S_{2k+1} = S_{2k-1} + R_k
// (the symmetric part of y drops out of I_k and the antisymmetric part out of R_k, because
// sin((P - n) theta) = sin(n theta) and the DFT kernels are odd or even about n = P / 2).
// Two real pencils y', y'' share one complex DFT of z = y' + i y'':
//   Y'_k = (Z_k + conj Z_{P-k}) / 2,   Y''_k = (Z_k - conj Z_{P-k}) / (2 i).
// P is prime in the paper's meshes (97, 73, 193: the transform-cost remark of Sec. 4.4), so
// the DFT of length P is Bluestein's chirp transform: with w_n = exp(i pi n^2 / P),
//   Z_k = conj(w_k) sum_n (z_n conj(w_n)) w_{k-n},
// a circular convolution of length L (a power of two >= 2P - 1) done as
// IFFT_L(FFT_L(z conj w) * FFT_L(b)), b_m = w_|m| for |m| < P (wrapped), FFT_L(b) tabulated
// on the host in FP64 (its product fused into the first stage of the inverse).  Each FFT_L
// is a Stockham transform in shared memory with radix-16 butterflies in registers
// (fft_util.cuh); R pencil pairs per CTA, R L = 4096 complex values per buffer.  FP32
// throughout.
//
// The six passes, their layouts and epilogues are those of the one-axis tensor-core passes:
// each reads rows whose transform axis is contiguous and writes its result transposed,
// out[k][row], so that the next pass again finds its axis contiguous; the third pass
// divides by lambda_l + lambda_m + lambda_n, the last scales by 8 / (Ng + 1)^3 and writes the
// padded potential.  Boxes of different Ng are served by one launch per pass: each group
// of boxes sharing Ng owns a range of the grid's CTAs.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "device_util.cuh"
#include "fft_util.cuh"

namespace scola {

namespace {

constexpr int kRxThreads = 256;
constexpr int kRxSpan = 4096;       // complex values per transform batch (R pairs x L)
constexpr int kMaxRxGroups = 4;     // Ng groups per launch (more: further launches)

enum RxPass { RX_F = 1, RX_XF = 2, RX_ZI = 3, RX_YI = 4, RX_XI = 5 };

struct RxGroupArgs {
    const Chunk *tiles;             // (box, tile of 2 R rows)
    int ntiles, cta_beg, cta_end;   // CTAs [cta_beg, cta_end) of the grid serve this group
    int Ng, P, L, logL, R;
    const float2 *w;                // w_n, n < P
    const float2 *Bk;               // FFT_L(b)
    const float2 *tw;               // exp(-2 pi i j / L), j < L
    const float2 *w256;             // the radix-16 second-stage twiddles
    const float *sn;                // sin(pi n / P), n < P
    const float *lam;               // Dirichlet eigenvalues, Ng
};

struct RxArgs {
    const BoxDesc *boxes;
    RxGroupArgs g[kMaxRxGroups];
    int ngroups;
    const float *in;
    float *out;
};

using fft::cmul;
using fft::cmulc;

// shared-memory buffer of the R rows of one transform batch (padded rows, odd stride)
int rx_buf(int L) { return (kRxSpan / L) * fft::row_stride(L, kRxSpan / L); }

// twiddles held in shared memory: L where a stage reads them, else none
int rx_tw(int L) { return fft::needs_tw(31 - __builtin_clz((unsigned)L)) ? L : 0; }

size_t rx_smem_bytes(int Ng, int P, int L) {
    return sizeof(float2) * ((size_t)2 * rx_buf(L) + fft::kW256 + rx_tw(L) + L + P) + sizeof(float) * ((size_t)P + Ng) +
           16;
}

template <int PASS>
__global__ void __launch_bounds__(kRxThreads, 3) k_dst_radix(const RxArgs A) {
    int gi = 0;
    while (gi + 1 < A.ngroups && (int)blockIdx.x >= A.g[gi].cta_end) ++gi;
    const RxGroupArgs &G = A.g[gi];
    if ((int)blockIdx.x < G.cta_beg || (int)blockIdx.x >= G.cta_end) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const int Ng = G.Ng, P = G.P, L = G.L, logL = G.logL, R = G.R;
    const int rows = 2 * R;                                // pencils per tile (a power of two)
    const int Ngs = Ng | 1;                                // odd row stride of the result rows
    const int Ls = fft::row_stride(L, R);                  // padded row stride of the transforms
    const int ntw = fft::needs_tw(logL) ? L : 0;
    float2 *buf0 = reinterpret_cast<float2 *>(smem);
    float2 *buf1 = buf0 + R * Ls;
    float2 *w256 = buf1 + R * Ls;                          // 256
    float2 *tw = w256 + fft::kW256;                        // L where read, else none
    float2 *Bk = tw + ntw;                                 // L
    float2 *w = Bk + L;                                    // P
    float *sn = reinterpret_cast<float *>(w + P);          // P
    float *lam = sn + P;                                   // Ng
    for (int q = threadIdx.x; q < ntw; q += kRxThreads) tw[q] = G.tw[q];
    for (int q = threadIdx.x; q < fft::kW256; q += kRxThreads) w256[q] = G.w256[q];
    for (int q = threadIdx.x; q < L; q += kRxThreads) Bk[q] = G.Bk[q];
    for (int q = threadIdx.x; q < P; q += kRxThreads) {
        w[q] = G.w[q];
        sn[q] = G.sn[q];
    }
    for (int q = threadIdx.x; q < Ng; q += kRxThreads) lam[q] = G.lam[q];
    __syncthreads();
    const long long Ng2 = (long long)Ng * Ng;
    const float scale = PASS == RX_XI ? 8.0f / ((float)(Ng + 1) * (Ng + 1) * (Ng + 1)) : 1.0f;
    const float invL = 1.0f / (float)L;
    const int H = P / 2;
    const int nstep = G.cta_end - G.cta_beg;
    for (int t = (int)blockIdx.x - G.cta_beg; t < G.ntiles; t += nstep) {
        const Chunk tl = G.tiles[t];
        const BoxDesc &B = A.boxes[tl.box];
        const long long row0 = (long long)tl.start * rows;
        const int nrow = (int)min((long long)rows, Ng2 - row0);
        // the tile's rows, contiguous in global memory, staged as floats in buf1 (rows past
        // the box's last are zero: the pair separation below needs finite partners)
        float *xs = reinterpret_cast<float *>(buf1);
        const float *src = A.in + B.m_off + row0 * Ng;
        for (int q = threadIdx.x; q < rows * Ng; q += kRxThreads) xs[q] = q < nrow * Ng ? src[q] : 0.0f;
        __syncthreads();
        // forward transform of a_n = (y'_n + i y''_n) conj(w_n) (n < P; zero to L), formed from
        // the staged rows as the first stage loads them
        auto chirped = [&](int pr, int n) {
            float2 v = make_float2(0.f, 0.f);
            if (n >= 1 && n < P) {
                const float *x1 = xs + (2 * pr) * Ng, *x2 = x1 + Ng;
                const float s = sn[n];
                const float a1 = x1[n - 1], b1 = x1[P - n - 1], a2 = x2[n - 1], b2 = x2[P - n - 1];
                const float y1 = s * (a1 + b1) + 0.5f * (a1 - b1);
                const float y2 = s * (a2 + b2) + 0.5f * (a2 - b2);
                v = cmulc(make_float2(y1, y2), w[n]);
            }
            return v;
        };
        float2 *f = fft::transform<-1>(chirped, buf0, buf1, R, logL, tw, w256);
        // inverse transform of its product with FFT_L(b)
        float2 *g = f == buf0 ? buf1 : buf0;
        const float2 *fc = f;
        auto product = [&](int pr, int n) { return cmul(fc[pr * Ls + fft::pad(n)], Bk[n]); };
        f = fft::transform<+1>(product, g, f, R, logL, tw, w256);
        // unpack the pairs: even outputs S_{2k} = -Im Y_k; odd increments R_k (R_0 / 2) placed
        // at the odd outputs' columns, summed below
        float *S = reinterpret_cast<float *>(f == buf0 ? buf1 : buf0);
        for (int q = threadIdx.x; q < R * (H + 1); q += kRxThreads) {
            const int pr = q / (H + 1), k = q - pr * (H + 1);
            const float2 *fr = f + pr * Ls;
            const int km = k == 0 ? 0 : P - k;
            float2 Zk = cmulc(fr[fft::pad(k)], w[k]), Zm = cmulc(fr[fft::pad(km)], w[km]);
            Zk.x *= invL; Zk.y *= invL; Zm.x *= invL; Zm.y *= invL;
            const float re1 = 0.5f * (Zk.x + Zm.x), im1 = 0.5f * (Zk.y - Zm.y);
            const float re2 = 0.5f * (Zk.y + Zm.y), im2 = -0.5f * (Zk.x - Zm.x);
            float *s1 = S + (2 * pr) * Ngs, *s2 = s1 + Ngs;
            if (k >= 1 && 2 * k <= Ng) {
                s1[2 * k - 1] = -im1;
                s2[2 * k - 1] = -im2;
            }
            if (2 * k + 1 <= Ng) {
                s1[2 * k] = k == 0 ? 0.5f * re1 : re1;
                s2[2 * k] = k == 0 ? 0.5f * re2 : re2;
            }
        }
        __syncthreads();
        // odd outputs: running sums of the increments along each row, one warp per row
        {
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            const int K = (Ng + 1) / 2, per = (K + 31) / 32;
            for (int r = warp; r < rows; r += kRxThreads / 32) {
                float *sr = S + r * Ngs;
                const int i0 = min(K, lane * per), i1 = min(K, i0 + per);
                float own = 0.0f;
                for (int i = i0; i < i1; ++i) own += sr[2 * i];
                float incl = own;
                for (int o = 1; o < 32; o <<= 1) {
                    const float u = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += u;
                }
                float acc = incl - own;
                for (int i = i0; i < i1; ++i) {
                    acc += sr[2 * i];
                    sr[2 * i] = acc;
                }
            }
        }
        __syncthreads();
        // out[k][row] (consecutive threads: consecutive rows)
        const int logrows = __ffs(rows) - 1;
        for (int q = threadIdx.x; q < Ng * rows; q += kRxThreads) {
            const int kk = q >> logrows, r = q & (rows - 1);
            if (r >= nrow) continue;
            const int row = (int)row0 + r;                  // < Ng^2 <= 2^16
            float v = S[r * Ngs + kk];
            const int rhi = row / Ng, rlo = row - rhi * Ng;
            if (PASS == RX_XI) {
                const int Gp = B.gpad;
                const long long Sd = Ng + 2 * Gp;
                A.out[B.pp_off + ((long long)(kk + Gp) * Sd + (rhi + Gp)) * Sd + (rlo + Gp)] = v * scale;
            } else {
                if (PASS == RX_XF) v = v / (lam[kk] + lam[rhi] + lam[rlo]);
                A.out[B.m_off + (long long)kk * Ng2 + row] = v;
            }
        }
        __syncthreads();
    }
}

template <int PASS>
cudaError_t set_rx_attr() {
    return cudaFuncSetAttribute(k_dst_radix<PASS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)rx_smem_bytes(256, 257, 1024));
}

// The groups a launch serves: the bound batch's (one per Ng), or the current box's alone in
// the per-tile form.
std::vector<RxGroup> rx_launch_groups(const Ctx &c) {
    std::vector<RxGroup> out;
    for (const RxGroup &G : c.rx_groups) {
        if (c.view_box >= 0) {
            if (G.Ng != c.boxes_h[c.view_box].Ng) continue;
            RxGroup V = G;
            V.tiles = c.rx_tiles + c.rx_tile_beg[c.view_box];
            V.ntiles = c.rx_tile_end[c.view_box] - c.rx_tile_beg[c.view_box];
            out.push_back(V);
        } else if (G.ntiles > 0) {
            out.push_back(G);
        }
    }
    return out;
}

template <int PASS>
cudaError_t run_rx_pass(Ctx &c, const float *in, float *out) {
    const std::vector<RxGroup> groups = rx_launch_groups(c);
    for (size_t g0 = 0; g0 < groups.size(); g0 += kMaxRxGroups) {
        const int ng = (int)std::min<size_t>(kMaxRxGroups, groups.size() - g0);
        RxArgs a;
        a.boxes = c.boxes;
        a.ngroups = ng;
        a.in = in;
        a.out = out;
        size_t smem = 0;
        double work = 0.0;
        for (int i = 0; i < ng; ++i) {
            const RxGroup &G = groups[g0 + i];
            smem = std::max(smem, rx_smem_bytes(G.Ng, G.P, G.L));
            work += (double)G.ntiles * G.R * G.L * G.logL;
        }
        int per_sm = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dst_radix<PASS>, kRxThreads, smem) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        const int slots = c.num_sms * per_sm;
        // CTAs split among the groups by their share of the butterflies (each at least one, at
        // most one per tile)
        int beg = 0;
        for (int i = 0; i < ng; ++i) {
            const RxGroup &G = groups[g0 + i];
            const double share = (double)G.ntiles * G.R * G.L * G.logL / work;
            const int n = std::max(1, std::min(G.ntiles, (int)std::lround(share * slots)));
            RxGroupArgs &q = a.g[i];
            q.tiles = G.tiles;
            q.ntiles = G.ntiles;
            q.cta_beg = beg;
            q.cta_end = beg + n;
            q.Ng = G.Ng;
            q.P = G.P;
            q.L = G.L;
            q.logL = G.logL;
            q.R = G.R;
            q.w = reinterpret_cast<const float2 *>(c.table_arena + G.w_off);
            q.Bk = reinterpret_cast<const float2 *>(c.table_arena + G.bk_off);
            q.tw = reinterpret_cast<const float2 *>(c.table_arena + G.tw_off);
            q.w256 = reinterpret_cast<const float2 *>(c.table_arena + c.fft_w256_off);
            q.sn = c.table_arena + G.sn_off;
            q.lam = c.table_arena + G.lam_off;
            beg += n;
        }
        k_dst_radix<PASS><<<beg, kRxThreads, smem, c.stream>>>(a);
        ++c.launches;
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

void rx_plan(int Ng, int &P, int &L, int &logL, int &R) {
    P = Ng + 1;
    L = 32;
    logL = 5;
    while (L < 2 * P - 1) {
        L <<= 1;
        ++logL;
    }
    R = kRxSpan / L;
}

bool rx_supported(int Ng) {
    if (Ng < 1) return false;
    int P, L, logL, R;
    rx_plan(Ng, P, L, logL, R);
    return R >= 1 && rx_smem_bytes(Ng, P, L) <= rx_smem_bytes(256, 257, 1024);
}

void rx_tables(RxGroup &G, std::vector<float> &arena) {
    rx_plan(G.Ng, G.P, G.L, G.logL, G.R);
    const int P = G.P, L = G.L;
    auto even = [&]() {
        if (arena.size() & 1) arena.push_back(0.0f);
        return (long long)arena.size();
    };
    // chirp w_n = exp(i pi n^2 / P) (phase reduced exactly: n^2 mod 2P)
    std::vector<double> wr(P), wi(P);
    for (int n = 0; n < P; ++n) {
        const long long e = ((long long)n * n) % (2LL * P);
        wr[n] = std::cos(M_PI * (double)e / P);
        wi[n] = std::sin(M_PI * (double)e / P);
    }
    G.w_off = even();
    for (int n = 0; n < P; ++n) {
        arena.push_back((float)wr[n]);
        arena.push_back((float)wi[n]);
    }
    // FFT_L of b (b_m = w_|m| for |m| < P, wrapped), a direct FP64 sum over a cosine table
    std::vector<double> br(L, 0.0), bi(L, 0.0), cs(L), sn(L);
    for (int m = 0; m < P; ++m) {
        br[m] = wr[m];
        bi[m] = wi[m];
        if (m > 0) {
            br[L - m] = wr[m];
            bi[L - m] = wi[m];
        }
    }
    for (int j = 0; j < L; ++j) {
        cs[j] = std::cos(2.0 * M_PI * j / L);
        sn[j] = std::sin(2.0 * M_PI * j / L);
    }
    G.bk_off = even();
    for (int k = 0; k < L; ++k) {
        double re = 0.0, im = 0.0;
        for (int m = 0; m < L; ++m) {
            if (br[m] == 0.0 && bi[m] == 0.0) continue;
            const int j = (int)(((long long)k * m) % L);      // exp(-2 pi i k m / L)
            re += br[m] * cs[j] + bi[m] * sn[j];
            im += bi[m] * cs[j] - br[m] * sn[j];
        }
        arena.push_back((float)re);
        arena.push_back((float)im);
    }
    G.tw_off = even();
    for (int j = 0; j < L; ++j) {
        arena.push_back((float)cs[j]);
        arena.push_back((float)-sn[j]);
    }
    G.sn_off = (long long)arena.size();
    for (int n = 0; n < P; ++n) arena.push_back((float)std::sin(M_PI * n / P));
}

cudaError_t init_rx_kernels() {
    cudaError_t e;
    if ((e = set_rx_attr<RX_F>())) return e;
    if ((e = set_rx_attr<RX_XF>())) return e;
    if ((e = set_rx_attr<RX_ZI>())) return e;
    if ((e = set_rx_attr<RX_YI>())) return e;
    return set_rx_attr<RX_XI>();
}

cudaError_t launch_poisson_rx_pass(Ctx &c, int pass) {
    // buffers: source (work2) -> work -> work2 -> work -> work2 -> work -> phi
    switch (pass) {
        case 0: return run_rx_pass<RX_F>(c, c.work2, c.work);
        case 1: return run_rx_pass<RX_F>(c, c.work, c.work2);
        case 2: return run_rx_pass<RX_XF>(c, c.work2, c.work);
        case 3: return run_rx_pass<RX_ZI>(c, c.work, c.work2);
        case 4: return run_rx_pass<RX_YI>(c, c.work2, c.work);
        case 5: return run_rx_pass<RX_XI>(c, c.work, c.phi);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_poisson_rx_buffers(Ctx &c, const float *in, float *w1, float *w2, float *out_pad) {
    cudaError_t e = run_rx_pass<RX_F>(c, in, w1);
    if (e == cudaSuccess) e = run_rx_pass<RX_F>(c, w1, w2);
    if (e == cudaSuccess) e = run_rx_pass<RX_XF>(c, w2, w1);
    if (e == cudaSuccess) e = run_rx_pass<RX_ZI>(c, w1, w2);
    if (e == cudaSuccess) e = run_rx_pass<RX_YI>(c, w2, w1);
    if (e == cudaSuccess) e = run_rx_pass<RX_XI>(c, w1, out_pad);
    return e;
}

}  // namespace scola
