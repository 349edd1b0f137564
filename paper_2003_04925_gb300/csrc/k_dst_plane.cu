// Dirichlet Poisson solve in three mesh passes on the tensor cores: the plane pass
// (App. C, Eqs. 63-71).
//
// The solve of a box mesh with Ng <= 96 and Ng % 4 == 0 runs as
//   pass 1  z+     the one-axis pass of k_dst_tc.cu:   src[i][j][k] -> W1[n][i][j]
//   pass 2  plane  this kernel: every z-frequency plane n of W1, held in shared memory, is
//                  transformed along y and x, divided by lambda_l + lambda_m + lambda_n, and
//                  transformed back along x and y                -> W2[n][i'][j']
//   pass 3  z-     the one-axis pass reading W2 plane by plane (k_dst_tc.cu, P_ZM), writing
//                  the padded potential in its natural [i][j][k] layout
// so the mesh crosses device memory three times per solve instead of six.
//
// Each step is D = S X^T with the sine matrix S (S_kn = sin(pi (k+1)(n+1)/(Ng+1))) as the
// M = 128 operand and the plane's Ng rows as the N operand, split into TF32 hi and lo parts
// (3xTF32, or four products with lo x lo).  S_hi and S_lo stay in tensor memory for the
// whole launch (the A operand of tcgen05.mma may come from TMEM), so an N = 96 MMA reads only
// the 3 KB data operand from shared memory: ~48 cycles against ~56 with both operands in
// shared memory, and the shared-memory bandwidth stays free for the epilogues.  TMEM lane u
// of D holds output index u of every row, so one epilogue thread per lane owns one row of
// the next step's operand: it reads its lane, splits it and writes it straight into the
// K-major operand in shared memory, and the next step contracts the other axis:
//   step 1  rows i,   K = j   ->  lanes m  (y frequency), columns i
//   step 2  rows m,   K = i   ->  lanes l  (x frequency), columns m   (then / lambda sum)
//   step 3  rows l,   K = m   ->  lanes j' (y),           columns l
//   step 4  rows j',  K = l   ->  lanes i' (x),           columns j'  -> row i' of W2[n]
// Three planes are in flight per CTA (three operand buffers, three accumulators): while
// the epilogues turn two planes' accumulators into their next operands, the tensor cores
// run the third plane's step, and the next plane's copy lands behind them.
//
// One persistent CTA per SM, 14 warps:
//   warps 4e .. 4e+3 (e = 0, 1, 2)  buffer e: split its planes into hi/lo, the epilogues of
//                                   their four steps
//   warp 12    TMEM allocation; lane 0 issues tcgen05.mma and tcgen05.commit
//   warp 13    lane 0 issues the tensor copies of each plane (Ng/32 boxes of 32 x Npad)
// The operands are K-major with the 128-byte swizzle (chunks of 32 columns).  The CTAs of
// a launch are split among the Ng groups of the boxes (as in k_dst_tc.cu).  Every wait is
// bounded (about 2 s); on expiry the CTA raises the error flag, stops issuing, waits
// (bounded) for its issued copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "device_util.cuh"
#include "tc_util.cuh"

namespace scola {

namespace {

using namespace tc;

constexpr int kPlThreads = 448;
constexpr int kPlBuf = 3;       // planes in flight
constexpr int kPlGroups = 4;

struct PlaneGroupArgs {
    CUtensorMap in_map;          // W1 as rows of Ng floats: boxes of 32 x Npad, 128-byte swizzle
    const Chunk *items;          // (box, plane n)
    const float *S;              // sine matrix rows, Ng x (32 nka) (the one-axis passes' table)
    const float *lam;            // Dirichlet eigenvalues, Ng
    int nitems, Ng, Npad, nka;   // nka: 32-column chunks of the sine matrix and of the operands
    int cta0, nctas;
};

struct PlaneArgs {
    PlaneGroupArgs grp[kPlGroups];
    int ngroups;
    const BoxDesc *boxes;
    float *out;
    int *err;
    int lo_lo;
};

// One epilogue thread's row after step STEP of a plane, accumulator chunks c0 .. c0 + 2 (v:
// 16 columns each; chunks >= nc16 absent).  Steps 1-3: the row of the next operand (K-major,
// 128-byte swizzle, hi and lo TF32 parts), zero outside the Ng x Ng block; step 2 first
// divides by the eigenvalue sum (row: x frequency l, column: y frequency m, plane: z
// frequency n).  Step 4: row i' of the output plane, written to global memory.
template <int STEP>
__device__ __forceinline__ void plane_rows(const float (&v)[3][16], int c0, int nc16, int row, int Ng, int Npad,
                                           uint32_t och, unsigned char *hi, unsigned char *lo, const float *lam,
                                           float lam_row, float lam_n, float *dst) {
    if (STEP == 4) {
        if (row >= Ng) return;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            const int c = c0 + cc;
            if (c >= nc16) break;
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                const int col = c * 16 + 4 * qq;
                if (col < Ng)
                    *reinterpret_cast<float4 *>(dst + col) =
                        make_float4(v[cc][4 * qq], v[cc][4 * qq + 1], v[cc][4 * qq + 2], v[cc][4 * qq + 3]);
            }
        }
        return;
    }
    if (row >= Npad) return;
    const bool rv = row < Ng;
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
        const int c = c0 + cc;
        if (c >= nc16) break;
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
            const int col0 = c * 16 + 4 * qq;
            float x[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                float y = v[cc][4 * qq + t];
                if (STEP == 2) y = __fdividef(y, lam_row + lam[col0 + t] + lam_n);
                x[t] = (rv && col0 + t < Ng) ? y : 0.0f;
            }
            const float4 h = make_float4(tf32_rn(x[0]), tf32_rn(x[1]), tf32_rn(x[2]), tf32_rn(x[3]));
            const uint32_t off = (uint32_t)(col0 >> 5) * och + sw128_offset(row, col0 & 31);
            *reinterpret_cast<float4 *>(hi + off) = h;
            *reinterpret_cast<float4 *>(lo + off) =
                make_float4(tf32_rn(x[0] - h.x), tf32_rn(x[1] - h.y), tf32_rn(x[2] - h.z), tf32_rn(x[3] - h.w));
        }
    }
}

__global__ void __launch_bounds__(kPlThreads, 1) k_dst_plane(const __grid_constant__ PlaneArgs A) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    int gi = 0;
    while (gi + 1 < A.ngroups && (int)blockIdx.x >= A.grp[gi + 1].cta0) ++gi;
    const PlaneGroupArgs &G = A.grp[gi];
    const int bid = (int)blockIdx.x - G.cta0, nbid = G.nctas;
    const int Ng = G.Ng, Npad = G.Npad, nka = G.nka;
    const int Kp = nka * 32;                                   // sine columns held (TMEM)
    const uint32_t och = (uint32_t)Npad * 128;                 // one operand chunk (32 K)
    const uint32_t bhalf = (uint32_t)nka * och;                // one operand, hi or lo
    // TMEM columns: S_hi [0, Kp), S_lo [Kp, 2 Kp), accumulator e at 2 Kp + e accw
    const uint32_t accw = (uint32_t)((Npad + 31) / 32 * 32);
    unsigned char *bufs = base;                                // buffer e: hi, then lo
    uint64_t *bars = (uint64_t *)(bufs + 2 * kPlBuf * (size_t)bhalf);
    uint64_t *loaded = bars;                 // the plane's tensor copies have landed
    uint64_t *opready = bars + kPlBuf;       // the next step's operand is written (128 arrivals)
    uint64_t *accfull = bars + 2 * kPlBuf;   // the step's MMAs are complete
    uint64_t *bufempty = bars + 3 * kPlBuf;  // step 4 is complete: the buffer may take the next plane
    uint64_t *drain = bars + 4 * kPlBuf;
    uint32_t *tmem_slot = (uint32_t *)(drain + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    float *lam = (float *)(tmem_slot + 4);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    // ---- set-up: eigenvalues, clean operand buffers, barriers, tensor memory
    for (int q = tid; q < 128; q += kPlThreads) lam[q] = q < Ng ? G.lam[q] : 0.0f;
    for (int q = tid; q < (int)(2 * kPlBuf * bhalf / 16); q += kPlThreads)
        reinterpret_cast<float4 *>(bufs)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    const long long my_items = G.nitems > bid ? (G.nitems - 1 - bid) / nbid + 1 : 0;
    if (tid == 0) {
        for (int e = 0; e < kPlBuf; ++e) {
            mbar_init(&loaded[e], 1);
            mbar_init(&opready[e], 128);
            mbar_init(&accfull[e], 1);
            mbar_init(&bufempty[e], 1);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 12) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (warp < 4) {
        // S into TMEM: lane k holds row k (zero for k >= Ng), hi parts in columns [0, Kp),
        // lo parts in [Kp, 2 Kp); the table row k has Kp columns, zero beyond Ng
        const int k = warp * 32 + lane;
        const uint32_t lb = (uint32_t)(warp * 32) << 16;
        for (int c = 0; c < Kp / 16; ++c) {
            float h[16], l[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float sv = k < Ng ? G.S[(long long)k * Kp + c * 16 + j] : 0.0f;
                h[j] = tf32_rn(sv);
                l[j] = tf32_rn(sv - h[j]);
            }
            tmem_st16(tmem + lb + (uint32_t)(c * 16), h);
            tmem_st16(tmem + lb + (uint32_t)(Kp + c * 16), l);
        }
        tmem_st_wait();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const long long Ng2 = (long long)Ng * Ng;
    const long long ntrip = (my_items + kPlBuf - 1) / kPlBuf;

    if (warp == 13) {
        // ---------------------------------------------------------------- tensor copies
        // plane p goes to buffer p % 3 once step 4 of plane p - 3 has finished with it; on an
        // abort, wait (bounded) for the copies already issued before the CTA may exit
        if (lane == 0) {
            long long p = 0;
            for (; p < my_items && !*abort_flag; ++p) {
                const int e = (int)(p % kPlBuf);
                const long long j = p / kPlBuf;
                if (j > 0 && !mbar_wait(&bufempty[e], (uint32_t)((j - 1) & 1), abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                const Chunk it = G.items[bid + p * nbid];
                const long long m_off = A.boxes[it.box].m_off;
                const int y = (int)(m_off / Ng + (long long)it.start * Ng);     // row (n, i = 0)
                unsigned char *hi = bufs + (size_t)e * 2 * bhalf;
                mbar_arrive_expect_tx(&loaded[e], bhalf);
                for (int c = 0; c < nka; ++c)
                    tma_load_2d(smem_u32(hi + (size_t)c * och), &G.in_map, c * 32, y, &loaded[e]);
            }
            if (*abort_flag) {
                const unsigned long long t0 = now_ns();
                for (long long q = p - kPlBuf > 0 ? p - kPlBuf : 0; q < p; ++q)
                    while (!mbar_try_wait(&loaded[q % kPlBuf], (uint32_t)((q / kPlBuf) & 1)) &&
                           now_ns() - t0 < kWaitNs) {
                    }
            }
        }
    } else if (warp == 12) {
        // ---------------------------------------------------------------- MMA issuer
        // order: for each triple of planes, steps 1..4, each step for the triple's planes
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(128, Npad);
            const bool lo_lo = A.lo_lo != 0;
            bool ok = true;
            for (long long q = 0; q < ntrip && ok && !*abort_flag; ++q)
                for (int s = 1; s <= 4 && ok; ++s)
                    for (int e = 0; e < kPlBuf; ++e) {
                        if (q * kPlBuf + e >= my_items) break;
                        if (!mbar_spin(&opready[e], (uint32_t)((s - 1) & 1), abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t d = tmem + (uint32_t)(2 * Kp) + (uint32_t)e * accw;
                        // descriptors advance by (byte offset >> 4) in their address field
                        // (shared addresses < 2^18: no carry out of the field)
                        const uint64_t bh0 = sw128_desc(smem_u32(bufs + (size_t)e * 2 * bhalf));
                        const uint64_t bl0 = bh0 + (bhalf >> 4);
                        for (int kc = 0; kc < nka; ++kc) {
                            const uint64_t bhc = bh0 + ((uint64_t)kc * (och >> 4)), blc = bl0 + ((uint64_t)kc * (och >> 4));
                            const uint32_t ahc = tmem + (uint32_t)(kc * 32), alc = ahc + (uint32_t)Kp;
                            if (lo_lo) {
#pragma unroll
                                for (int kk = 0; kk < 4; ++kk) {
                                    if (kc * 32 + kk * 8 >= Ng) break;
                                    const uint64_t bhi = bhc + (uint64_t)(kk * 2), blo = blc + (uint64_t)(kk * 2);
                                    mma_tf32_ts(d, ahc + kk * 8, bhi, idesc, (kc | kk) ? 1u : 0u);
                                    mma_tf32_ts(d, ahc + kk * 8, blo, idesc, 1);
                                    mma_tf32_ts(d, alc + kk * 8, bhi, idesc, 1);
                                    mma_tf32_ts(d, alc + kk * 8, blo, idesc, 1);
                                }
                            } else {
#pragma unroll
                                for (int kk = 0; kk < 4; ++kk) {
                                    if (kc * 32 + kk * 8 >= Ng) break;
                                    const uint64_t bhi = bhc + (uint64_t)(kk * 2), blo = blc + (uint64_t)(kk * 2);
                                    mma_tf32_ts(d, ahc + kk * 8, bhi, idesc, (kc | kk) ? 1u : 0u);
                                    mma_tf32_ts(d, ahc + kk * 8, blo, idesc, 1);
                                    mma_tf32_ts(d, alc + kk * 8, bhi, idesc, 1);
                                }
                            }
                        }
                        mma_commit(&accfull[e]);
                        if (s == 4) mma_commit(&bufempty[e]);
                    }
            if (!ok) *abort_flag = 1;
        }
    } else {
        // ---------------------------------------------------------------- warps 0-11
        // warp group e = warp / 4 serves buffer e (planes p = 3 q + e); warp w reads TMEM
        // lanes 32 (w & 3) + lane, the output index of its row, over all column chunks
        const int e = warp >> 2, lq = warp & 3;
        const int gt = tid & 127;                       // thread within the group
        const int row = lq * 32 + lane;
        unsigned char *hi = bufs + (size_t)e * 2 * bhalf, *lo = hi + bhalf;
        const uint32_t tb = tmem + (uint32_t)(2 * Kp) + (uint32_t)e * accw + ((uint32_t)(lq * 32) << 16);
        const int nc16 = Npad / 16;                     // 16-column accumulator chunks (<= 6)
        bool ok = true;
        for (long long q = 0; q < ntrip && ok && !*abort_flag; ++q) {
            const long long p = q * kPlBuf + e;
            if (p >= my_items) break;
            const Chunk it = G.items[bid + p * nbid];
            const int n = it.start;
            const long long m_off = A.boxes[it.box].m_off;
            // split the loaded plane in place: hi over the copy, lo into the other half; rows
            // >= Ng (the next plane's rows brought by the box) are cleared.  Four 16-byte units
            // per thread in flight at a time
            if (!mbar_spin(&loaded[e], (uint32_t)(q & 1), abort_flag)) {
                ok = false;
                break;
            }
            const int units = nka * Npad * 8;
            for (int u0 = gt; u0 < units; u0 += 4 * 128) {
                float4 v[4];
                uint32_t off[4];
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int u = u0 + 128 * b;
                    const int c = u / (Npad * 8), rem = u - c * (Npad * 8);
                    const int r = rem >> 3, qq = rem & 7;
                    off[b] = (uint32_t)c * och + sw128_offset(r, 4 * qq);
                    v[b] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (u < units && r < Ng) v[b] = *reinterpret_cast<const float4 *>(hi + off[b]);
                }
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    if (u0 + 128 * b >= units) break;
                    const float4 h = make_float4(tf32_rn(v[b].x), tf32_rn(v[b].y), tf32_rn(v[b].z), tf32_rn(v[b].w));
                    *reinterpret_cast<float4 *>(hi + off[b]) = h;
                    *reinterpret_cast<float4 *>(lo + off[b]) = make_float4(
                        tf32_rn(v[b].x - h.x), tf32_rn(v[b].y - h.y), tf32_rn(v[b].z - h.z), tf32_rn(v[b].w - h.w));
                }
            }
            fence_proxy_async();
            mbar_arrive(&opready[e]);
            const float lam_row = row < Ng ? lam[row] : 0.0f, lam_n = lam[n];
            float *dst = A.out + m_off + (long long)n * Ng2 + (long long)row * Ng;
            for (int s = 1; s <= 4; ++s) {
                if (!mbar_spin(&accfull[e], (uint32_t)((s - 1) & 1), abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // the lane's columns in two halves of up to three 16-column chunks, each half's
                // TMEM loads in flight together
                for (int c0 = 0; c0 < nc16; c0 += 3) {
                    float v[3][16];
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc)
                        if (c0 + cc < nc16) tmem_ld16_issue(tb + (uint32_t)((c0 + cc) * 16), v[cc]);
                    tmem_ld_wait();
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) tmem_regs_ready(v[cc]);
                    if (s == 1) plane_rows<1>(v, c0, nc16, row, Ng, Npad, och, hi, lo, lam, lam_row, lam_n, dst);
                    else if (s == 2) plane_rows<2>(v, c0, nc16, row, Ng, Npad, och, hi, lo, lam, lam_row, lam_n, dst);
                    else if (s == 3) plane_rows<3>(v, c0, nc16, row, Ng, Npad, och, hi, lo, lam, lam_row, lam_n, dst);
                    else plane_rows<4>(v, c0, nc16, row, Ng, Npad, och, hi, lo, lam, lam_row, lam_n, dst);
                }
                if (s < 4) fence_proxy_async();
                tc_fence_before();
                if (s < 4) mbar_arrive(&opready[e]);
            }
        }
        if (!ok) *abort_flag = 1;
    }

    // ---- tear-down: every role has left its loop; drain, then free tensor memory
    if (warp == 12 && lane == 0 && *abort_flag) {
        mma_commit(drain);
        const unsigned long long t0 = now_ns();
        while (!mbar_try_wait(drain, 0) && now_ns() - t0 < kWaitNs) {
        }
    }
    if (*abort_flag && tid == 0) atomicOr(A.err, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 12) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

size_t plane_smem_bytes(int Ng, int Npad, int nka) {
    (void)Ng;
    return 1024 + 2 * kPlBuf * (size_t)nka * Npad * 128 + (4 * kPlBuf + 1) * 8 + 16 + 128 * 4 + 64;
}

constexpr size_t kPlSmemBudget = 227 * 1024;

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// W1 as a 2D tensor of rows of Ng floats, boxes of 32 x Npad with the 128-byte swizzle of
// the MMA's K-major operand.
cudaError_t plane_map(Ctx &c, const float *buf, int Ng, int Npad, CUtensorMap *out) {
    static EncodeTiledFn encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return e != cudaSuccess ? e : cudaErrorNotSupported;
        encode = (EncodeTiledFn)fn;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)Ng, (cuuint64_t)(c.M / Ng)};
    const cuuint64_t strides[1] = {(cuuint64_t)Ng * sizeof(float)};
    const cuuint32_t box[2] = {32u, (cuuint32_t)Npad};
    const cuuint32_t estr[2] = {1, 1};
    if (encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(buf), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

}  // namespace

bool plane_supported(int Ng) {
    if (Ng < 8 || Ng > 96 || Ng % 4 != 0) return false;
    const int Npad = (Ng + 15) / 16 * 16, nka = (Ng + 31) / 32;
    return plane_smem_bytes(Ng, Npad, nka) <= kPlSmemBudget;
}

cudaError_t init_plane_kernel() {
    return cudaFuncSetAttribute(k_dst_plane, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPlSmemBudget);
}

// The plane pass over the given Ng groups (at most kPlGroups per launch): items are (box,
// plane) pairs of every box of each group; the persistent grid is split among the groups in
// proportion to their work (planes x Ng^2).
cudaError_t launch_plane_pass(Ctx &c, const std::vector<TcGroup> &groups, const float *in, float *out) {
    for (size_t g0 = 0; g0 < groups.size(); g0 += kPlGroups) {
        const int ng = (int)std::min(groups.size() - g0, (size_t)kPlGroups);
        PlaneArgs a;
        std::memset(&a, 0, sizeof(a));
        double total = 0;
        std::vector<double> work(ng);
        for (int g = 0; g < ng; ++g) {
            const TcGroup &G = groups[g0 + g];
            work[g] = (double)G.nplanes * G.Ng * G.Ng;
            total += work[g];
        }
        int cta0 = 0;
        size_t smem = 0;
        for (int g = 0; g < ng; ++g) {
            const TcGroup &G = groups[g0 + g];
            PlaneGroupArgs &P = a.grp[g];
            P.Ng = G.Ng;
            P.Npad = (G.Ng + 15) / 16 * 16;
            P.nka = G.nkc;
            cudaError_t e = plane_map(c, in, P.Ng, P.Npad, &P.in_map);
            if (e != cudaSuccess) return e;
            P.items = G.planes;
            P.nitems = G.nplanes;
            P.S = c.table_arena + G.s_off;
            P.lam = c.table_arena + G.lam_off;
            int n = (int)(c.num_sms * work[g] / std::max(total, 1.0));
            n = std::max(1, std::min(n, std::max(1, G.nplanes)));
            if (g == ng - 1) n = std::max(1, std::min(std::max(1, c.num_sms - cta0), std::max(1, G.nplanes)));
            P.cta0 = cta0;
            P.nctas = n;
            cta0 += n;
            smem = std::max(smem, plane_smem_bytes(P.Ng, P.Npad, P.nka));
        }
        a.ngroups = ng;
        a.boxes = c.boxes;
        a.out = out;
        a.err = c.dev_err;
        a.lo_lo = c.tc_lo_lo ? 1 : 0;
        k_dst_plane<<<cta0, kPlThreads, smem, c.stream>>>(a);
        ++c.launches;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace scola
