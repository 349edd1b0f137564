// Dirichlet Poisson solve on the 5th-generation tensor cores (App. C, Eqs. 62-71).
//
// The 3D DST-I is applied as six dense pencil products D = A S^T (S_kn =
// sin(pi (k+1)(n+1)/(Ng+1)), symmetric), each on rows whose transform axis is
// contiguous in memory.  Every pass writes its result transposed,
// out[col][row], so that the next pass again finds its axis contiguous:
//
//   pass  input rows (axis)    k    writes              epilogue
//   z+    src[i][j][k]  (i,j)  k    W1[n][i][j]         (src: delta' from the deposit)
//   y+    W1[n][i][j]   (n,i)  j    W2[m][n][i]
//   x+    W2[m][n][i]   (m,n)  i    W3[l][m][n]         / (lambda_l + lambda_m + lambda_n)
//   z-    W3[l][m][n]   (l,m)  n    W4[k'][l][m]
//   y-    W4[k'][l][m]  (k',l) m    W5[j'][k'][l]
//   x-    W5[j'][k'][l] (j',k') l   Phi[i'+2][j'+2][k'+2]   * 8 / (Ng+1)^3
//
// Precision: FP32 operands split as a = a_hi + a_lo with a_hi the value with
// its 13 low mantissa bits cleared (exact in TF32); D accumulates
// a_hi s_hi + a_hi s_lo + a_lo s_hi in FP32 in tensor memory (3xTF32), and
// a_lo s_lo as well in the four-product form.  A single TF32 product gives
// position errors of ~0.1 PM cell over a run, the three-term form stays near
// the FP32 level.
//
// One persistent CTA per SM, 13 warps:
//   warps 0-7  epilogue: tcgen05.ld of the accumulator (warp w reads TMEM lanes
//              32(w%4)..+31 = tile rows, half of the columns), scaling, transposed
//              global stores
//   warps 8-11 producer: cp.async copies of 128-row x 32-column chunks into a
//              ring of raw staging buffers, DEPTH chunks ahead; each thread then
//              splits the bytes it copied into hi/lo and stores them in the
//              128-byte-swizzled K-major layout of the MMA stage
//   warp 12    TMEM allocation; lane 0 issues tcgen05.mma and tcgen05.commit
// Stages of A chunks form a ring guarded by full/empty mbarriers; the
// accumulator is double buffered in TMEM (tmem_full / tmem_empty).  Every
// wait is bounded (about 2 s of %globaltimer); on expiry the CTA raises an
// error flag in global memory, stops issuing work, waits for its issued
// tensor-core work to drain, frees its tensor memory and returns.
#include <stdint.h>

#include <algorithm>

#include "device_util.cuh"

namespace scola {

namespace {

constexpr int kTM = 128;             // rows per tile (MMA M)
constexpr int kKC = 32;              // K per chunk (one 128-byte swizzle atom of FP32)
constexpr int kChunkBytes = kTM * 128;
constexpr int kThreads = 416;          // 8 epilogue, 4 producer, 1 MMA warps
constexpr int kMaxGroups = 4;          // 16-column TMEM groups per epilogue warp (Npad <= 128)
constexpr unsigned long long kWaitNs = 2000000000ull;

enum TcPass { P_F = 1, P_XF = 2, P_ZI = 3, P_YI = 4, P_XI = 5 };   // P_F: z+ and y+

// Per-CTA cache of the tiles a CTA processes (the first kTileCache of them): the box
// offsets and the first row, so that the producer and the epilogue need no dependent
// global loads per tile.
struct TileInfo {
    long long m_off, pp_off;
    int row0, pad;
};
constexpr int kTileCache = 192;

struct TcArgs {
    const BoxDesc *boxes;
    const Chunk *tiles;          // (box, tile-in-box)
    int ntiles;
    int Ng, Npad, nkc, nstage;   // uniform Ng for the launch; nstage = hi/lo MMA stages
    const float *S;              // FP32 sine matrix, Npad x (nkc*32), zero padded
    const float *lam;            // Dirichlet eigenvalues, Ng
    const float *in;
    float *out;
    int *err;
    int lo_lo;                   // 1: also accumulate a_lo s_lo (four TF32 products)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase; false on timeout or when another role aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    const unsigned long long t0 = now_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 63) {
            if (*abort_flag) return false;
            if (now_ns() - t0 > kWaitNs) return false;
        }
    }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;              // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;    // stride byte offset
    d |= (uint64_t)1u << 46;              // descriptor version
    d |= (uint64_t)2u << 61;              // 128-byte swizzle
    return d;
}

// Instruction descriptor: D F32, A and B TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 16 columns of this warp's 32 TMEM lanes into v, without waiting for them.
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, float (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
          "=f"(v[7]), "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]),
          "=f"(v[14]), "=f"(v[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Orders later uses of v after a tcgen05.wait::ld (the registers become valid there).
__device__ __forceinline__ void tmem_regs_ready(float (&v)[16]) {
    asm volatile(""
                 : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]),
                   "+f"(v[7]), "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]), "+f"(v[12]), "+f"(v[13]),
                   "+f"(v[14]), "+f"(v[15]));
}

// Byte offset of element (r, k) (k within the 32-wide chunk) in a 128B-swizzled K-major tile.
__device__ __forceinline__ uint32_t sw128_offset(int r, int k) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 2) ^ (r & 7)) & 7) << 4) + (k & 3) * 4);
}

__device__ __forceinline__ float tf32_hi(float x) {
    return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

template <int PASS, int DEPTH>
__global__ void __launch_bounds__(kThreads, 1) k_dst_tc(TcArgs A) {
    constexpr int RS = DEPTH + 1;                   // raw staging ring
    constexpr int RAWB = kChunkBytes;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-aligned (in the shared window) base for the swizzled operand tiles
    unsigned char *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int Ng = A.Ng, Npad = A.Npad, nkc = A.nkc, NST = A.nstage;
    const int sbytes = nkc * Npad * 128;            // one of S_hi / S_lo
    unsigned char *S_hi = base;
    unsigned char *S_lo = base + sbytes;
    unsigned char *stages = base + 2 * sbytes;      // NST x (A_hi chunk, A_lo chunk)
    unsigned char *raw = stages + (size_t)NST * 2 * kChunkBytes;   // RS raw chunks
    uint64_t *bars = (uint64_t *)(raw + (size_t)RS * RAWB);
    uint64_t *full = bars;
    uint64_t *empty = bars + NST;
    uint64_t *tfull = bars + 2 * NST;
    uint64_t *tempty = bars + 2 * NST + 2;
    uint64_t *drain = bars + 2 * NST + 4;
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * NST + 5);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    float *lam = (float *)(tmem_slot + 4);
    TileInfo *tinfo = (TileInfo *)(base + ((((unsigned char *)(lam + Ng) - base) + 15) & ~15));

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    // ---- set-up: S (hi/lo split, swizzled), lambda, barriers, tensor memory
    const int Kp = nkc * kKC;
    for (int q = tid; q < Npad * Kp; q += kThreads) {
        const int n = q / Kp, k = q % Kp;
        const float s = A.S[q];
        const float hi = tf32_hi(s);
        const uint32_t off = (uint32_t)(k / kKC) * (Npad * 128) + sw128_offset(n, k % kKC);
        *(float *)(S_hi + off) = hi;
        *(float *)(S_lo + off) = s - hi;
    }
    for (int q = tid; q < Ng; q += kThreads) lam[q] = A.lam[q];
    const long long my_tiles = A.ntiles > (int)blockIdx.x ? (A.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto load_tile = [&](long long k) {
        const Chunk tl = A.tiles[(int)blockIdx.x + k * (int)gridDim.x];
        TileInfo ti;
        ti.m_off = A.boxes[tl.box].m_off;
        ti.pp_off = A.boxes[tl.box].pp_off;
        ti.row0 = tl.start * kTM;
        ti.pad = 0;
        return ti;
    };
    for (int k = tid; k < my_tiles && k < kTileCache; k += kThreads) tinfo[k] = load_tile(k);
    auto tile_at = [&](long long k) { return k < kTileCache ? tinfo[k] : load_tile(k); };
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 128);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 256);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 12) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const long long Ng2 = (long long)Ng * Ng;

    if (warp >= 8 && warp < 12) {
        // ---------------------------------------------------------------- producer
        // chunk g of this CTA = tile (blockIdx.x + (g / nkc) gridDim.x), K-chunk g % nkc.
        // Thread pt copies and later converts items q = pt + 128 e (e < 8): row q >> 3,
        // float4 group q & 7 of the chunk.
        const int pt = tid - 256;
        const uint32_t raw_s = smem_u32(raw);
        const long long nchunks = my_tiles * nkc;
        auto issue = [&](long long g) {
            if (g < nchunks) {
                const int c = (int)(g % nkc);
                const TileInfo ti = tile_at(g / nkc);
                const long long m_off = ti.m_off;
                const int row0 = ti.row0;
                const uint32_t dst0 = raw_s + (uint32_t)((g % RS) * RAWB);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int q = pt + 128 * e;
                    const int r = q >> 3, kq = q & 7;
                    const int k = c * kKC + kq * 4;
                    const int R = row0 + r;
                    const bool ok = (long long)R < Ng2 && k < Ng;
                    const float *src = A.in + m_off + (ok ? (long long)R * Ng + k : 0);
                    cp_async16(dst0 + sw128_offset(r, kq * 4), src, ok ? 16u : 0u);
                }
            }
            cp_async_commit();
        };
        for (int d = 0; d < DEPTH; ++d) issue(d);
        for (long long g = 0; g < nchunks && !*abort_flag; ++g) {
            issue(g + DEPTH);
            cp_async_wait<DEPTH>();
            const int s = (int)(g % NST);
            if (!mbar_wait(&empty[s], (uint32_t)(((g / NST) & 1) ^ 1), abort_flag)) {
                *abort_flag = 1;
                break;
            }
            unsigned char *ah = stages + (size_t)s * 2 * kChunkBytes;
            unsigned char *al = ah + kChunkBytes;
            const unsigned char *rw = raw + (size_t)(g % RS) * RAWB;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int q = pt + 128 * e;
                const int r = q >> 3, kq = q & 7;
                const uint32_t off = sw128_offset(r, kq * 4);
                const float4 v = *reinterpret_cast<const float4 *>(rw + off);
                const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
                const float4 l = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
                *reinterpret_cast<float4 *>(ah + off) = h;
                *reinterpret_cast<float4 *>(al + off) = l;
            }
            fence_proxy_async();
            mbar_arrive(&full[s]);
        }
        cp_async_wait<0>();
    } else if (warp == 12) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(kTM, Npad);
            uint32_t g = 0, t = 0;
            for (int it = blockIdx.x; it < A.ntiles && !*abort_flag; it += gridDim.x, ++t) {
                const int a = t & 1;
                if (!mbar_wait(&tempty[a], ((t >> 1) & 1) ^ 1, abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(a * 128);
                bool ok = true;
                for (int c = 0; c < nkc; ++c, ++g) {
                    const int s = g % NST;
                    if (!mbar_wait(&full[s], (g / NST) & 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t ah = smem_u32(stages + (size_t)s * 2 * kChunkBytes);
                    const uint32_t al = ah + kChunkBytes;
                    const uint32_t bh = smem_u32(S_hi) + (uint32_t)(c * Npad * 128);
                    const uint32_t bl = smem_u32(S_lo) + (uint32_t)(c * Npad * 128);
                    const int ksteps = min(kKC, Ng - c * kKC + 7) / 8;   // skip all-zero K steps
                    for (int kk = 0; kk < ksteps; ++kk) {
                        const uint32_t o = (uint32_t)kk * 32;
                        mma_tf32(d, sw128_desc(ah + o), sw128_desc(bh + o), idesc, (c | kk) != 0);
                        mma_tf32(d, sw128_desc(ah + o), sw128_desc(bl + o), idesc, 1);
                        mma_tf32(d, sw128_desc(al + o), sw128_desc(bh + o), idesc, 1);
                        if (A.lo_lo) mma_tf32(d, sw128_desc(al + o), sw128_desc(bl + o), idesc, 1);
                    }
                    mma_commit(&empty[s]);
                }
                if (!ok) {
                    *abort_flag = 1;
                    break;
                }
                mma_commit(&tfull[a]);
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue (warps 0-7)
        // warp w reads TMEM lanes 32 (w & 3) .. + 31 (its tile rows) and the 16-column groups
        // g = (w >> 2) + 2 i: all its groups are loaded before one wait, then the accumulator
        // is released and the stores follow.
        const int quarter = warp & 3, half = warp >> 2;
        const int row_in_tile = quarter * 32 + lane;
        const int ngroups = Npad / 16;
        const float scale = (PASS == P_XI) ? 8.0f / ((float)(Ng + 1) * (Ng + 1) * (Ng + 1)) : 1.0f;
        uint32_t t = 0;
        for (int it = blockIdx.x; it < A.ntiles && !*abort_flag; it += gridDim.x, ++t) {
            const int a = t & 1;
            if (!mbar_wait(&tfull[a], (t >> 1) & 1, abort_flag)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint32_t tbase = tmem + (uint32_t)(a * 128) + ((uint32_t)(quarter * 32) << 16);
            float v[kMaxGroups][16];
#pragma unroll
            for (int i = 0; i < kMaxGroups; ++i)
                if (half + 2 * i < ngroups) tmem_ld16_issue(tbase + (uint32_t)(16 * (half + 2 * i)), v[i]);
            tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < kMaxGroups; ++i) tmem_regs_ready(v[i]);
            tc_fence_before();
            mbar_arrive(&tempty[a]);
            const TileInfo ti = tile_at(t);
            const int Ri = ti.row0 + row_in_tile;
            if ((long long)Ri >= Ng2) continue;
            const int rhi = Ri / Ng, rlo = Ri - rhi * Ng;
            float lsum = 0.0f;
            if (PASS == P_XF) lsum = lam[rhi] + lam[rlo];
            // element (row Ri, column col) goes to base + col * cstride
            float *base;
            long long cstride;
            if (PASS == P_XI) {
                const long long S = Ng + 4;
                base = A.out + ti.pp_off + (2 * S + (rhi + 2)) * S + (rlo + 2);
                cstride = S * S;
            } else {
                base = A.out + ti.m_off + Ri;
                cstride = Ng2;
            }
#pragma unroll
            for (int i = 0; i < kMaxGroups; ++i) {
                const int c0 = 16 * (half + 2 * i);
                if (c0 >= Ng) break;
                float *p = base + (long long)c0 * cstride;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = c0 + j;
                    if (col >= Ng) break;
                    float x = v[i][j];
                    if (PASS == P_XI) x *= scale;
                    if (PASS == P_XF) x = __fdividef(x, lam[col] + lsum);
                    *p = x;
                    p += cstride;
                }
            }
        }
    }

    // ---- tear-down: every role has left its loop; drain, then free tensor memory
    if (warp == 12 && lane == 0 && *abort_flag) {
        // wait (bounded) until every MMA this thread issued has finished writing TMEM
        mma_commit(drain);
        const unsigned long long t0 = now_ns();
        while (!mbar_try_wait(drain, 0) && now_ns() - t0 < kWaitNs) {
        }
    }
    if (*abort_flag && tid == 0) atomicExch(A.err, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 12) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

size_t tc_smem_bytes(int Npad, int nkc, int nstage, int Ng, int raw_bytes) {
    return 1024 + 2 * (size_t)nkc * Npad * 128 + (size_t)nstage * 2 * kChunkBytes + (size_t)raw_bytes +
           (2 * nstage + 5) * 8 + 16 + (size_t)Ng * 4 + 16 + kTileCache * sizeof(TileInfo) + 64;
}

constexpr size_t kSmemBudget = 227 * 1024;
constexpr int kDeep = 4, kShallow = 1;

// Deepest raw ring (DEPTH chunks ahead) that fits next to S and the MMA stages.
int pick_depth(const TcGroup &G) {
    if (tc_smem_bytes(G.Npad, G.nkc, G.nstage, G.Ng, (kDeep + 1) * kChunkBytes) <= kSmemBudget)
        return kDeep;
    return kShallow;
}

template <int PASS>
cudaError_t run_tc_pass(Ctx &c, const TcGroup &G, const float *in, float *out) {
    const int depth = pick_depth(G);
    TcArgs a;
    a.boxes = c.boxes;
    a.tiles = G.tiles;
    a.ntiles = G.ntiles;
    a.Ng = G.Ng;
    a.Npad = G.Npad;
    a.nkc = G.nkc;
    a.nstage = G.nstage;
    a.S = c.table_arena + G.s_off;
    a.lam = c.table_arena + G.lam_off;
    a.in = in;
    a.out = out;
    a.err = c.dev_err;
    a.lo_lo = c.tc_lo_lo ? 1 : 0;
    const size_t smem = tc_smem_bytes(G.Npad, G.nkc, G.nstage, G.Ng, (depth + 1) * kChunkBytes);
    const int grid = std::max(1, std::min(G.ntiles, c.num_sms));
    if (depth == kDeep)
        k_dst_tc<PASS, kDeep><<<grid, kThreads, smem, c.stream>>>(a);
    else
        k_dst_tc<PASS, kShallow><<<grid, kThreads, smem, c.stream>>>(a);
    ++c.launches;
    return cudaGetLastError();
}

}  // namespace

int tc_plan_stages(int Ng, int &Npad, int &nkc) {
    // two hi/lo MMA stages; the raw ring takes what is left (at least 2 chunks)
    Npad = ((Ng + 15) / 16) * 16;
    nkc = (Ng + kKC - 1) / kKC;
    const int nst = 2;
    if (tc_smem_bytes(Npad, nkc, nst, Ng, (kShallow + 1) * kChunkBytes) > kSmemBudget) return 0;
    return nst;
}

bool tc_supported(int Ng) {
    int Npad, nkc;
    return Ng >= 4 && Ng <= 128 && Ng % 4 == 0 && tc_plan_stages(Ng, Npad, nkc) >= 2;
}

template <int PASS>
cudaError_t set_tc_attr() {
    const int lim = (int)kSmemBudget;
    cudaError_t e = cudaFuncSetAttribute(k_dst_tc<PASS, kDeep>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_dst_tc<PASS, kShallow>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

cudaError_t init_tc_kernels() {
    cudaError_t e;
    if ((e = set_tc_attr<P_F>())) return e;
    if ((e = set_tc_attr<P_XF>())) return e;
    if ((e = set_tc_attr<P_ZI>())) return e;
    if ((e = set_tc_attr<P_YI>())) return e;
    return set_tc_attr<P_XI>();
}

// The launch groups: every Ng group, or in the per-tile form only the current box's tiles.
std::vector<TcGroup> active_groups(const Ctx &c) {
    if (c.view_box < 0) return c.tc_groups;
    std::vector<TcGroup> one;
    for (const TcGroup &G : c.tc_groups) {
        if (G.Ng != c.boxes_h[c.view_box].Ng) continue;
        TcGroup V = G;
        V.tiles = c.tc_tiles + c.tc_tile_beg[c.view_box];
        V.ntiles = c.tc_tile_end[c.view_box] - c.tc_tile_beg[c.view_box];
        one.push_back(V);
    }
    return one;
}

cudaError_t launch_poisson_tc_pass(Ctx &c, int pass) {
    // buffers: source (work2) -> work -> work2 -> work -> work2 -> work -> phi
    cudaError_t e = cudaSuccess;
    for (const TcGroup &G : active_groups(c)) {
        switch (pass) {
            case 0: e = run_tc_pass<P_F>(c, G, c.work2, c.work); break;
            case 1: e = run_tc_pass<P_F>(c, G, c.work, c.work2); break;
            case 2: e = run_tc_pass<P_XF>(c, G, c.work2, c.work); break;
            case 3: e = run_tc_pass<P_ZI>(c, G, c.work, c.work2); break;
            case 4: e = run_tc_pass<P_YI>(c, G, c.work2, c.work); break;
            case 5: e = run_tc_pass<P_XI>(c, G, c.work, c.phi); break;
            default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_poisson_tc(Ctx &c) {
    for (int p = 0; p < 6; ++p) {
        cudaError_t e = launch_poisson_tc_pass(c, p);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
// (launch_poisson in k_pm.cu uses the same sequence through launch_poisson_buffers.)

cudaError_t launch_poisson_tc_buffers(Ctx &c, const float *in, float *w1, float *w2, float *out_pad) {
    cudaError_t e = cudaSuccess;
    for (const TcGroup &G : active_groups(c)) {
        e = run_tc_pass<P_F>(c, G, in, w1);
        if (e == cudaSuccess) e = run_tc_pass<P_F>(c, G, w1, w2);
        if (e == cudaSuccess) e = run_tc_pass<P_XF>(c, G, w2, w1);
        if (e == cudaSuccess) e = run_tc_pass<P_ZI>(c, G, w1, w2);
        if (e == cudaSuccess) e = run_tc_pass<P_YI>(c, G, w2, w1);
        if (e == cudaSuccess) e = run_tc_pass<P_XI>(c, G, w1, out_pad);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace scola
