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
// M = 128 operand and the plane's Ng rows as the N operand, both split into FP16 hi and lo
// parts: S_hi X_hi + S_hi X_lo + S_lo X_hi (or four products with lo x lo) on
// tcgen05.mma kind::f16, which runs at twice the TF32 rate and reads half the operand
// bytes.  FP16 has TF32's 11-bit significand but a narrow exponent range, so every operand
// row (one pencil) is multiplied by a power of two 2^s that puts its largest magnitude in
// [2^14, 2^15) before the split, and S by 2^14: hi + lo then keep ~22 bits of the pencil
// relative to its largest element, as 3xTF32 does, smaller elements keep their absolute
// error at that level, and no part overflows.  Column n of D carries the factor
// 2^(14 + s_n) of pencil n; the epilogue that reads D multiplies it out (exactly) before it
// scales its own row.  S_hi and S_lo stay in tensor memory for the whole launch (the A
// operand of tcgen05.mma may come from TMEM), so the MMAs read only the data operand from
// shared memory.  TMEM lane u of D holds output index u of every row, so one epilogue thread
// per lane owns one row of the next step's operand: it reads its lane, scales and splits it
// and writes it straight into the K-major operand in shared memory, and the next step
// contracts the other axis:
//   step 1  rows i,   K = j   ->  lanes m  (y frequency), columns i
//   step 2  rows m,   K = i   ->  lanes l  (x frequency), columns m   (then / lambda sum)
//   step 3  rows l,   K = m   ->  lanes j' (y),           columns l
//   step 4  rows j',  K = l   ->  lanes i' (x),           columns j'  -> row i' of W2[n]
// The output plane is written row by row into the group's operand buffer (free once the
// step-4 MMAs are complete; the staging layout) and leaves by tensor store.
// Three planes are in flight per CTA (three operand buffers, three accumulators): while
// the epilogues turn two planes' accumulators into their next operands, the tensor cores
// run the third plane's step.  The FP32 planes land in two staging buffers by tensor copy;
// the group that takes a plane scales and splits it row by row into its operand buffer.
//
// One persistent CTA per SM, 11 warps (at most 168 registers a thread):
//   warps 4e .. 4e+2 (e = 0, 1, 2)  buffer e: split its planes into hi/lo, the epilogues of
//                                   their four steps (TMEM lanes 0 .. 95: Npad <= 96)
//   warp 7     TMEM allocation; lane 0 issues tcgen05.mma and tcgen05.commit
//   warp 3     lane 0 issues the tensor copies of each plane (Ng/32 boxes of 32 x Npad)
// The operands are K-major with the 128-byte swizzle (chunks of 64 FP16 columns; the
// staging buffers in chunks of 32 FP32 columns).  The CTAs of a launch are split among the
// Ng groups of the boxes (as in k_dst_tc.cu).  Every wait is bounded (about 2 s); on expiry
// the CTA raises the error flag, stops issuing, waits (bounded) for its issued copies and
// MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "device_util.cuh"
#include "tc_util.cuh"

namespace scola {

namespace {

using namespace tc;

constexpr int kPlThreads = 352;
constexpr int kPlRows = 96;    // threads of an epilogue group: one per operand row
constexpr int kPlBuf = 3;       // planes in flight
constexpr int kPlStage = 2;     // FP32 staging buffers for the tensor copies
constexpr int kPlGroups = 4;
constexpr int kPlMaxN = 96;     // largest Ng of the plane pass
constexpr int kSExp = 14;       // S is held as S 2^14
constexpr int kSCols = 64;      // TMEM columns of S_hi (two FP16 elements per column)

struct PlaneGroupArgs {
    CUtensorMap in_map;          // W1 as rows of Ng floats: boxes of 32 x Npad, 128-byte swizzle
    CUtensorMap out_map;         // W2 as rows of Ng floats: boxes of 32 x Ng, 128-byte swizzle
    const Chunk *items;          // (box, plane n)
    const float *S;              // sine matrix rows, Ng x (32 nka) (the one-axis passes' table)
    const float *lam;            // Dirichlet eigenvalues, Ng
    int nitems, Ng, Npad, nka;   // nka: 32-column chunks of the FP32 rows and of the sine table
    int cta0, nctas;
};

struct PlaneArgs {
    PlaneGroupArgs grp[kPlGroups];
    int ngroups;
    const BoxDesc *boxes;
    int *err;
    int lo_lo;
};

// 2^s as a float, |s| <= 126.
__device__ __forceinline__ float pow2f(int s) { return __uint_as_float((uint32_t)(127 + s) << 23); }

// The exponent s that puts a row's largest magnitude m in [2^14, 2^15): 0 for a zero or
// non-finite row, at most 100 (rows below 2^-86 keep their absolute error far below 2^-40).
__device__ __forceinline__ int row_exp(float m) {
    if (!(m > 0.0f) || !(m <= 3.0e38f)) return 0;
    const int E = (int)((__float_as_uint(m) >> 23) & 0xFFu) - 127;
    return min(kSExp - E, 100);
}

__device__ __forceinline__ uint32_t h2_bits(__half2 h) {
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}

// Row `row` of a K-major FP16 operand pair (128-byte swizzle, 64-column chunks och bytes
// apart): x[k] sc split into hi and lo, in units of 8 columns up to nu.
__device__ __forceinline__ void put_row(const float (&x)[kPlMaxN / 16][16], float sc, int row, int nu, uint32_t och,
                                        unsigned char *hi, unsigned char *lo) {
#pragma unroll
    for (int u = 0; u < kPlMaxN / 8; ++u) {
        if (u >= nu) break;
        uint32_t h[4], l[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float a = x[u >> 1][8 * (u & 1) + 2 * t] * sc, b = x[u >> 1][8 * (u & 1) + 2 * t + 1] * sc;
            const __half2 hh = __floats2half2_rn(a, b);
            const float2 hf = __half22float2(hh);
            h[t] = h2_bits(hh);
            l[t] = h2_bits(__floats2half2_rn(a - hf.x, b - hf.y));
        }
        const uint32_t off = (uint32_t)(u >> 3) * och + (uint32_t)((row >> 3) * 1024 + (row & 7) * 128) +
                             ((uint32_t)((u & 7) ^ (row & 7)) << 4);
        *reinterpret_cast<uint4 *>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4 *>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// Largest magnitude of a row: 16 independent partial maxima, then a tree (a short
// dependency chain instead of one of 96 steps).
__device__ __forceinline__ float row_max(const float (&x)[kPlMaxN / 16][16]) {
    float m[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) m[j] = fabsf(x[0][j]);
#pragma unroll
    for (int c = 1; c < kPlMaxN / 16; ++c)
#pragma unroll
        for (int j = 0; j < 16; ++j) m[j] = fmaxf(m[j], fabsf(x[c][j]));
#pragma unroll
    for (int w = 8; w > 0; w >>= 1)
#pragma unroll
        for (int j = 0; j < w; ++j) m[j] = fmaxf(m[j], m[j + w]);
    return m[0];
}

__global__ void __launch_bounds__(kPlThreads, 1) k_dst_plane(const __grid_constant__ PlaneArgs A) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    int gi = 0;
    while (gi + 1 < A.ngroups && (int)blockIdx.x >= A.grp[gi + 1].cta0) ++gi;
    const PlaneGroupArgs &G = A.grp[gi];
    const int bid = (int)blockIdx.x - G.cta0, nbid = G.nctas;
    const int Ng = G.Ng, Npad = G.Npad, nka = G.nka;
    const int Kp = nka * 32;                                   // columns of the sine table rows
    const int nk16 = (Ng + 15) / 16;                           // K steps of the MMAs
    const uint32_t och = (uint32_t)Npad * 128;                 // one 128-byte-wide chunk of rows
    const uint32_t bhalf = (uint32_t)((nk16 + 3) / 4) * och;   // one FP16 operand, hi or lo
    const uint32_t bstage = (uint32_t)nka * och;               // one FP32 staging buffer
    // TMEM columns: S_hi [0, 64), S_lo [64, 128), accumulator e at 128 + e accw
    const uint32_t accw = (uint32_t)((Npad + 31) / 32 * 32);
    unsigned char *ops = base;                                 // buffer e: hi, then lo
    unsigned char *stage = ops + 2 * kPlBuf * (size_t)bhalf;   // staging buffer b
    uint64_t *bars = (uint64_t *)(stage + kPlStage * (size_t)bstage);
    // loaded[e]: the copies of group e's next plane have landed.  The barrier belongs to the
    // consuming group, not to the staging buffer, so that its phases follow the group's own
    // planes (a buffer's planes alternate between groups, and a parity wait must never be
    // two phases ahead of the barrier)
    uint64_t *loaded = bars;
    uint64_t *stfree = bars + kPlBuf;                  // staging b: its plane is split (96 arrivals)
    uint64_t *opready = stfree + kPlStage;             // the next step's operand is written (96 arrivals)
    uint64_t *accfull = opready + kPlBuf;              // the step's MMAs are complete
    uint64_t *outw = accfull + kPlBuf;                 // the output plane is in shared memory (96 arrivals)
    uint64_t *outfree = outw + kPlBuf;                 // its tensor store has read it
    uint64_t *drain = outfree + kPlBuf;
    uint32_t *tmem_slot = (uint32_t *)(drain + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    float *lam = (float *)(tmem_slot + 4);
    float *uns = lam + 128;                            // [buffer][slot][column]: 2^-(14 + s) of row
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    // ---- set-up: eigenvalues, clean operand buffers, barriers, tensor memory
    for (int q = tid; q < 128; q += kPlThreads) lam[q] = q < Ng ? G.lam[q] : 0.0f;
    for (int q = tid; q < kPlBuf * 2 * 128; q += kPlThreads) uns[q] = 0.0f;
    for (int q = tid; q < (int)(2 * kPlBuf * bhalf / 16); q += kPlThreads)
        reinterpret_cast<float4 *>(ops)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    const long long my_items = G.nitems > bid ? (G.nitems - 1 - bid) / nbid + 1 : 0;
    if (tid == 0) {
        for (int b = 0; b < kPlStage; ++b) mbar_init(&stfree[b], kPlRows);
        for (int e = 0; e < kPlBuf; ++e) {
            mbar_init(&loaded[e], 1);
            mbar_init(&opready[e], kPlRows);
            mbar_init(&accfull[e], 1);
            mbar_init(&outw[e], kPlRows);
            mbar_init(&outfree[e], 1);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 7) {
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
        // S 2^14 into TMEM: lane k holds row k (zero for k >= Ng), two FP16 elements per
        // column (element 2c in the low half of column c), hi parts in columns [0, 64), lo
        // parts in [64, 128); the table row k has Kp columns, zero beyond Ng.  Warp w writes
        // lanes 32 w .. 32 w + 31
        const int k = warp * 32 + lane;
        const uint32_t lb = (uint32_t)(warp * 32) << 16;
        const float ss = pow2f(kSExp);
        for (int g = 0; g < kSCols / 16; ++g) {
            float h[16], l[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int c0 = 32 * g + 2 * j;
                const float a = (k < Ng && c0 < Kp) ? G.S[(long long)k * Kp + c0] * ss : 0.0f;
                const float b = (k < Ng && c0 + 1 < Kp) ? G.S[(long long)k * Kp + c0 + 1] * ss : 0.0f;
                const __half2 hh = __floats2half2_rn(a, b);
                const float2 hf = __half22float2(hh);
                h[j] = __uint_as_float(h2_bits(hh));
                l[j] = __uint_as_float(h2_bits(__floats2half2_rn(a - hf.x, b - hf.y)));
            }
            tmem_st16(tmem + lb + (uint32_t)(g * 16), h);
            tmem_st16(tmem + lb + (uint32_t)(kSCols + g * 16), l);
        }
        tmem_st_wait();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const long long ntrip = (my_items + kPlBuf - 1) / kPlBuf;

    if (warp == 3) {
        // ---------------------------------------------------------------- tensor copies
        // plane p goes to staging buffer p % 2 once plane p - 2 has been split out of it, and
        // completes on loaded[p % 3]; the copies are issued in plane order, so group p % 3 has
        // taken its plane p - 3 before plane p can land.  On an abort, wait (bounded) for the
        // copies already issued before the CTA may exit
        if (lane == 0) {
            long long p = 0;
            for (; p < my_items && !*abort_flag; ++p) {
                const int b = (int)(p % kPlStage);
                const long long j = p / kPlStage;
                if (j > 0 && !mbar_wait(&stfree[b], (uint32_t)((j - 1) & 1), abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                const Chunk it = G.items[bid + p * nbid];
                const long long m_off = A.boxes[it.box].m_off;
                const int y = (int)(m_off / Ng + (long long)it.start * Ng);     // row (n, i = 0)
                unsigned char *st = stage + (size_t)b * bstage;
                uint64_t *bar = &loaded[p % kPlBuf];
                mbar_arrive_expect_tx(bar, bstage);
                for (int c = 0; c < nka; ++c) tma_load_2d(smem_u32(st + (size_t)c * och), &G.in_map, c * 32, y, bar);
            }
            if (*abort_flag) {
                const unsigned long long t0 = now_ns();
                for (long long q = p - kPlStage > 0 ? p - kPlStage : 0; q < p; ++q)
                    while (!mbar_try_wait(&loaded[q % kPlBuf], (uint32_t)((q / kPlBuf) & 1)) &&
                           now_ns() - t0 < kWaitNs) {
                    }
            }
        }
    } else if (warp == 7) {
        // ---------------------------------------------------------------- MMA issuer
        // order: for each triple of planes, steps 1..4, each step for the triple's planes
        if (lane == 0) {
            const uint32_t idesc = idesc_f16(128, Npad);
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
                        const uint32_t d = tmem + (uint32_t)(2 * kSCols) + (uint32_t)e * accw;
                        // descriptors advance by (byte offset >> 4) in their address field
                        // (shared addresses < 2^18: no carry out of the field); a K step of 16
                        // FP16 columns is 32 bytes of the swizzled row, 8 TMEM columns of S
                        const uint64_t bh0 = sw128_desc(smem_u32(ops + (size_t)e * 2 * bhalf));
                        const uint64_t bl0 = bh0 + (bhalf >> 4);
                        for (int t = 0; t < nk16; ++t) {
                            const uint64_t off = (uint64_t)(t >> 2) * (och >> 4) + (uint64_t)((t & 3) * 2);
                            const uint32_t ah = tmem + (uint32_t)(t * 8), al = ah + (uint32_t)kSCols;
                            mma_f16_ts(d, ah, bh0 + off, idesc, t ? 1u : 0u);
                            mma_f16_ts(d, ah, bl0 + off, idesc, 1);
                            mma_f16_ts(d, al, bh0 + off, idesc, 1);
                            if (lo_lo) mma_f16_ts(d, al, bl0 + off, idesc, 1);
                        }
                        mma_commit(&accfull[e]);
                    }
            if (!ok) *abort_flag = 1;
        }
    } else {
        // ---------------------------------------------------------------- warps 4e .. 4e+2
        // warp group e = warp / 4 serves buffer e (planes p = 3 q + e); warp w reads TMEM
        // lanes 32 (w & 3) + lane, the output index of its row, over all column chunks.  Each
        // scheduler runs one warp of every group, so the groups wait with suspending waits
        // that leave the issue slots to the group at work
        const int e = warp >> 2, lq = warp & 3;
        const int row = lq * 32 + lane;
        unsigned char *hi = ops + (size_t)e * 2 * bhalf, *lo = hi + bhalf;
        float *un = uns + e * 2 * 128;
        const uint32_t tb = tmem + (uint32_t)(2 * kSCols) + (uint32_t)e * accw + ((uint32_t)(lq * 32) << 16);
        const int nc16 = Npad / 16;                     // 16-column accumulator chunks (<= 6)
        const int nu = 2 * nk16;                        // 8-column operand units written per row
        bool ok = true;
        for (long long q = 0; q < ntrip && ok && !*abort_flag; ++q) {
            const long long p = q * kPlBuf + e;
            if (p >= my_items) break;
            const Chunk it = G.items[bid + p * nbid];
            const int n = it.start;
            const long long m_off = A.boxes[it.box].m_off;
            const int b = (int)(p % kPlStage);
            if (!mbar_wait(&loaded[e], (uint32_t)(q & 1), abort_flag)) {
                ok = false;
                break;
            }
            float x[kPlMaxN / 16][16];
            {
                // the thread's row of the FP32 plane (rows >= Ng: the next plane's rows brought by
                // the copy, cleared; columns >= Ng: zero, filled by the copy beyond the tensor's
                // rows of Ng floats), then the staging buffer is released
                const unsigned char *st = stage + (size_t)b * bstage;
#pragma unroll
                for (int c = 0; c < kPlMaxN / 32; ++c)
#pragma unroll
                    for (int qq = 0; qq < 8; ++qq) {
                        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (c < nka && row < Ng)
                            v = *reinterpret_cast<const float4 *>(st + (uint32_t)c * och + sw128_offset(row, 4 * qq));
                        const int k = 32 * c + 4 * qq;
                        x[k >> 4][(k & 15)] = v.x;
                        x[k >> 4][(k & 15) + 1] = v.y;
                        x[k >> 4][(k & 15) + 2] = v.z;
                        x[k >> 4][(k & 15) + 3] = v.w;
                    }
                mbar_arrive(&stfree[b]);
                // the operand buffer holds the previous plane's output until its tensor store
                // has read it (issued by the group's thread 0, which signals here)
                if (q > 0) {
                    if (row == 0) {
                        bulk_wait_read();
                        mbar_arrive(&outfree[e]);
                    }
                    if (!mbar_wait(&outfree[e], (uint32_t)((q - 1) & 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                }
                const int s0 = row_exp(row_max(x));
                if (row < Npad) put_row(x, pow2f(s0), row, nu, och, hi, lo);
                un[row] = pow2f(-(kSExp + s0));
            }
            fence_proxy_async();
            mbar_arrive(&opready[e]);
            const float lam_row = row < Ng ? lam[row] : 0.0f, lam_n = lam[n];
            for (int s = 1; s <= 4; ++s) {
                if (!mbar_wait(&accfull[e], (uint32_t)((s - 1) & 1), abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int c = 0; c < kPlMaxN / 16; ++c)
                    if (c < nc16) tmem_ld16_issue(tb + (uint32_t)(c * 16), x[c]);
                tmem_ld_wait();
#pragma unroll
                for (int c = 0; c < kPlMaxN / 16; ++c) {
                    tmem_regs_ready(x[c]);
                    if (c >= nc16)
#pragma unroll
                        for (int j = 0; j < 16; ++j) x[c][j] = 0.0f;
                }
                // column k of D carries 2^(14 + s_k) of the row it came from (slot (s - 1) & 1);
                // step 2 divides by the eigenvalue sum (row: x frequency l, column: y frequency
                // m, plane: z frequency n).  D is exactly zero outside the Ng x Ng block (rows:
                // S is zero beyond Ng; columns: so are the operand rows), and so is y there
                // (lambda is zero-padded and lambda_n > 0); chunks >= nc16 are not loaded: zero
                const float4 *u_in = reinterpret_cast<const float4 *>(un + ((s - 1) & 1) * 128);
                const float4 *lam4 = reinterpret_cast<const float4 *>(lam);
#pragma unroll
                for (int c = 0; c < kPlMaxN / 16; ++c)
#pragma unroll
                    for (int jq = 0; jq < 4; ++jq) {
                        const float4 u4 = u_in[4 * c + jq];
                        const float uu[4] = {u4.x, u4.y, u4.z, u4.w};
                        float ll[4] = {0.f, 0.f, 0.f, 0.f};
                        if (s == 2) {
                            const float4 l4 = lam4[4 * c + jq];
                            ll[0] = l4.x, ll[1] = l4.y, ll[2] = l4.z, ll[3] = l4.w;
                        }
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const int j = 4 * jq + t;
                            float y = x[c][j] * uu[t];
                            if (s == 2) y = __fdividef(y, lam_row + ll[t] + lam_n);
                            x[c][j] = y;
                        }
                    }
                if (s == 4) {
                    // row i' of the output plane into the operand buffer (32-column chunks,
                    // 128-byte swizzle, as the copies bring the planes in); thread 0 of the
                    // group stores the plane once every row is written
                    if (row < Ng) {
#pragma unroll
                        for (int c = 0; c < kPlMaxN / 32; ++c)
#pragma unroll
                            for (int qq = 0; qq < 8; ++qq) {
                                const int k = 32 * c + 4 * qq;
                                if (c < nka)
                                    *reinterpret_cast<float4 *>(hi + (uint32_t)c * och + sw128_offset(row, 4 * qq)) =
                                        make_float4(x[k >> 4][k & 15], x[k >> 4][(k & 15) + 1], x[k >> 4][(k & 15) + 2],
                                                    x[k >> 4][(k & 15) + 3]);
                            }
                    }
                    fence_proxy_async();
                    tc_fence_before();
                    mbar_arrive(&outw[e]);
                    if (row == 0) {
                        if (!mbar_wait(&outw[e], (uint32_t)(q & 1), abort_flag)) {
                            ok = false;
                            break;
                        }
                        const int y = (int)(m_off / Ng + (long long)n * Ng);     // row (n, i' = 0)
                        for (int c = 0; c < nka; ++c) tma_store_2d(&G.out_map, c * 32, y, smem_u32(hi + (size_t)c * och));
                        bulk_commit();
                    }
                } else {
                    const int sr = row_exp(row_max(x));
                    if (row < Npad) put_row(x, pow2f(sr), row, nu, och, hi, lo);
                    un[(s & 1) * 128 + row] = pow2f(-(kSExp + sr));
                    fence_proxy_async();
                    tc_fence_before();
                    mbar_arrive(&opready[e]);
                }
            }
        }
        // thread 0's tensor stores complete before the CTA exits
        if (row == 0) bulk_wait_all();
        if (!ok) *abort_flag = 1;
    }

    // ---- tear-down: every role has left its loop; drain, then free tensor memory
    if (warp == 7 && lane == 0 && *abort_flag) {
        mma_commit(drain);
        const unsigned long long t0 = now_ns();
        while (!mbar_try_wait(drain, 0) && now_ns() - t0 < kWaitNs) {
        }
    }
    if (*abort_flag && tid == 0) atomicOr(A.err, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 7) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

size_t plane_smem_bytes(int Ng, int Npad, int nka) {
    const size_t nk64 = (size_t)(Ng + 63) / 64;
    return 1024 + 2 * kPlBuf * nk64 * Npad * 128 + kPlStage * (size_t)nka * Npad * 128 +
           (kPlStage + 5 * kPlBuf + 1) * 8 + 16 + 128 * 4 + kPlBuf * 2 * 128 * 4 + 64;
}

constexpr size_t kPlSmemBudget = 227 * 1024;

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// A plane-major mesh buffer as a 2D tensor of rows of Ng floats, boxes of 32 x `rows` with
// the 128-byte swizzle: W1 with rows = Npad (the staging layout the splitting threads read),
// W2 with rows = Ng (the output planes).
cudaError_t plane_map(Ctx &c, const float *buf, int Ng, int rows, CUtensorMap *out) {
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
    const cuuint32_t box[2] = {32u, (cuuint32_t)rows};
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
            if (e == cudaSuccess) e = plane_map(c, out, P.Ng, P.Ng, &P.out_map);
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
