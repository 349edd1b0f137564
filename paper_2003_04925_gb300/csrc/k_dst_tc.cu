// Dirichlet Poisson solve on the 5th-generation tensor cores (App. C, Eqs. 62-71).
//
// The 3D DST-I is applied as six dense pencil products over rows whose transform
// axis is contiguous in memory.  For a tile of 256 such rows X (256 x Ng) a pass
// computes D^T = S X^T on the tensor cores (S_kn = sin(pi (k+1)(n+1)/(Ng+1)),
// symmetric): the sine matrix is the M = 128 operand (rows n < Ng, resident in
// shared memory for the whole launch) and the data rows are the N = 256 operand, so
// every MMA instruction runs at the full N width of the tensor pipe.  TMEM lane n of
// the accumulator holds output column n for all 256 rows, and each epilogue thread
// writes contiguous runs of out[n][row]: every pass stores its result transposed,
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
// Precision: FP32 operands split as a = a_hi + a_lo, a_hi the nearest TF32 value and
// a_lo the nearest TF32 value of the remainder (together ~24 significant bits); D
// accumulates s_hi x_hi + s_hi x_lo + s_lo x_hi in FP32 in tensor memory (3xTF32), and
// s_lo x_lo as well in the four-product form.  A single TF32 product gives position
// errors of ~0.1 PM cell over a run, the three-term form stays near the FP32 level.
//
// Any Ng up to 256.  Meshes whose rows are 16-byte pitched (Ng % 4 == 0; folded: Ng % 32 == 0)
// reach the stages by TMA.  Other meshes (the paper's own geometry, Ng = Np,sCOLA + 1, Sec. 4
// Table 1) take the "ragged" path: the converter warps read each chunk from global memory with
// plain coalesced loads (rows beyond the box and columns beyond Ng read as zero) and write the
// split straight into the stage, and the epilogue stores element by element.
//
// Meshes with Ng > 128 use the mirror symmetry of the sine matrix,
// S_{k, Ng-1-n} = (-1)^k S_kn: the even outputs are the half-size product of the even rows
// of S with u_n = x_n + x_{Ng-1-n}, the odd outputs that of the odd rows with
// v_n = x_n - x_{Ng-1-n} (n < Ng/2).  For odd Ng the middle element pairs with itself: u
// takes 2 x_mid there, so the even-parity matrix holds half of that column, and the odd
// outputs do not see it (their sine vanishes there).  Each work item is one parity of one
// tile: the CTA holds that parity's matrix (ceil(Ng/2) rows and columns for the even outputs,
// floor(Ng/2) for the odd ones, at most 128), loads
// every 16-column chunk of the rows together with its mirror chunk, and its converters
// form u or v and split it into hi and lo parts in place of the two loaded chunks.  Half
// the products of the direct form, and the two
// items of a tile run on neighbouring CTAs at the same time, so the second read of the
// rows comes from L2.
//
// One persistent CTA per SM, 18 warps:
//   warps 0-7  epilogue: tcgen05.ld of the accumulator (warp w reads TMEM lanes
//              32(w%4)..+31 = output columns, half of the 256 rows), a 32 x 32
//              transpose through shared memory, scaling, coalesced global stores
//   warps 8-15 converters: split each landed stage in place into its hi and lo parts
//   warp 16    TMEM allocation; lane 0 issues tcgen05.mma and tcgen05.commit
//   warp 17    lane 0 issues the tensor copies (TMA) of 256-row x 16-column chunks of
//              the data into a ring of MMA stages (64-byte-swizzled K-major)
// Stages form a ring guarded by full/empty mbarriers; the accumulator is double
// buffered in TMEM (tmem_full / tmem_empty, 2 x 256 columns).  Every wait is
// bounded (about 2 s of %globaltimer); on expiry the CTA raises an error flag in
// global memory, stops issuing work, waits for its issued tensor-core work to
// drain, frees its tensor memory and returns.
#include <cuda.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "device_util.cuh"
#include "tc_util.cuh"

namespace scola {

namespace {

using namespace tc;

constexpr int kTM = 128;             // MMA M: rows of the sine matrix (output index n < Ng <= 128)
constexpr int kTN = kTcTileRows;     // MMA N: data rows per tile (256)
constexpr int kKA = 32;              // K per sine-matrix chunk (one 128-byte swizzle row of FP32)
constexpr int kKB = 16;              // K per data chunk (one 64-byte swizzle row of FP32)
constexpr int kHalfBytes = kTN * 64; // one data chunk, hi or lo (16 KB)
constexpr int kThreads = 576;        // 8 epilogue, 8 converter, 1 MMA, 1 TMA warps
constexpr int kProducers = 256;      // converter threads; each splits kHalfBytes / 16 / kProducers units per chunk
constexpr int kUnits = kHalfBytes / 16 / kProducers;
constexpr int kTmemCols = 2 * kTN;   // double-buffered accumulator

// Per epilogue warp: a 32 x 33 float block for transposing 32 columns x 32 rows.
constexpr int kXposeBytes = 32 * 33 * 4;

enum TcPass { P_F = 1, P_XF = 2, P_ZI = 3, P_YI = 4, P_XI = 5, P_ZM = 6 };   // P_F: z+ and y+
// P_ZM: the z inverse of the three-pass solve (k_dst_plane.cu), reading W2[n][i][j] plane by
// plane: a tile is 256 consecutive cells q = (i, j) of the planes, its K chunk 16 planes n;
// the tensor copy brings the [16 n][256 q] box unswizzled, the converters transpose it into
// the K-major operand while splitting it, and the epilogue writes the padded potential in
// its natural layout, one TMEM lane (output k) per consecutive float, so 32 lanes store 128
// contiguous bytes.

// Stage bytes of a pass: hi and lo halves (and the untransposed copy for P_ZM).
__host__ __device__ constexpr int stage_bytes(int pass) { return (pass == P_ZM ? 3 : 2) * kHalfBytes; }

// Per-CTA cache of the tiles a CTA processes (the first kTileCache of them): the box
// offsets and the first row, so that the producer and the epilogue need no dependent
// global loads per tile.
struct TileInfo {
    long long m_off, pp_off;
    int row0, pad;
};
constexpr int kTileCache = 96;

// One Ng group of a launch: the boxes sharing Ng, their tiles, tables and tensor map, and
// the CTAs [cta0, cta0 + nctas) that process them.  Every CTA holds the sine matrix of its
// own group only, so boxes of uneven mesh sizes share one launch per pass.
struct TcGroupArgs {
    CUtensorMap in_map;          // the input as rows of Ng floats (64-byte swizzle boxes 16 x 256)
    const Chunk *tiles;          // (box, tile-in-box)
    const float *S;              // FP32 sine matrix, Npad x (nkc*32), zero padded (folded: the
                                 // even-row and then the odd-row half matrices)
    const float *lam;            // Dirichlet eigenvalues, Ng
    int ntiles;                  // work items: tiles, or 2 x tiles (one per parity) when folded
    int Ng, Npad, nkc, nstage;   // nkc sine chunks; nstage data stages
    int ragged;                  // 1: rows not 16-byte pitched; plain loads and stores (no TMA)
    int cta0, nctas;             // this group's CTAs (an even count when folded)
};
constexpr int kMaxTcGroups = 4;

struct TcArgs {
    TcGroupArgs grp[kMaxTcGroups];
    int ngroups;
    const BoxDesc *boxes;
    const float *in;
    float *out;
    int *err;
    int lo_lo;                   // 1: also accumulate a_lo s_lo (four TF32 products)
    unsigned long long stall_ns; // failure-detection self-test: > 0 makes the MMA thread first wait
                                 // this long on a barrier nothing arrives on, then abort
};

template <int PASS, bool FOLD>
__global__ void __launch_bounds__(kThreads, 1) k_dst_tc(const __grid_constant__ TcArgs A) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-aligned (in the shared window) base for the swizzled operand tiles
    unsigned char *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    // this CTA's group, and its index among the group's CTAs
    int gi = 0;
    while (gi + 1 < A.ngroups && (int)blockIdx.x >= A.grp[gi + 1].cta0) ++gi;
    const TcGroupArgs &G = A.grp[gi];
    const int bid = (int)blockIdx.x - G.cta0, nbid = G.nctas;
    const int Ng = G.Ng, nka = G.nkc, NST = G.nstage;
    // folded: this CTA's parity (the group's CTA count is even, so item b + k nbid keeps the
    // parity of b), and the contraction length and matrix rows Nk = Ng / 2
    const int parity = FOLD ? (bid & 1) : 0;
    const int Nk = FOLD ? (parity ? Ng / 2 : (Ng + 1) / 2) : Ng;
    const int nkb = (Nk + kKB - 1) / kKB;                 // data chunks per tile
    const uint32_t sch = (uint32_t)((Nk + 7) / 8) * 1024; // one sine chunk (hi or lo), Nk rows
    // The M = 128 operand reads 128 rows from each sine chunk; rows >= Ng come from what
    // follows (the next chunk, or the stages) and only feed TMEM lanes that are never read.
    unsigned char *S_hi = base;
    unsigned char *S_lo = base + nka * sch;
    constexpr int SB = stage_bytes(PASS);
    unsigned char *stages = base + 2 * nka * sch;
    float *xpose = (float *)(stages + (size_t)NST * SB);              // 8 x kXposeBytes (not P_ZM)
    uint64_t *bars = (uint64_t *)((unsigned char *)xpose + (PASS == P_ZM ? 0 : 8 * kXposeBytes));
    uint64_t *full = bars;                 // converted (MMA may read the stage)
    uint64_t *empty = bars + NST;          // consumed (the stage may be reloaded)
    uint64_t *loaded = bars + 2 * NST;     // the tensor copy into the stage has landed
    uint64_t *tfull = bars + 3 * NST;
    uint64_t *tempty = bars + 3 * NST + 2;
    uint64_t *drain = bars + 3 * NST + 4;
    uint32_t *tmem_slot = (uint32_t *)(bars + 3 * NST + 5);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    float *lam = (float *)(tmem_slot + 4);
    TileInfo *tinfo = (TileInfo *)(base + ((((unsigned char *)(lam + Ng) - base) + 15) & ~15));

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    // ---- set-up: S (hi/lo split, swizzled), lambda, tile table, barriers, tensor memory
    const int Kp = nka * kKA;
    const float *Sg = G.S + (FOLD ? (long long)parity * G.Npad * Kp : 0LL);
    for (int q = tid; q < Nk * Kp; q += kThreads) {
        const int n = q / Kp, k = q % Kp;
        const float sv = Sg[q];
        const float hi = tf32_rn(sv);
        const uint32_t off = (uint32_t)(k / kKA) * sch + sw128_offset(n, k % kKA);
        *(float *)(S_hi + off) = hi;
        *(float *)(S_lo + off) = tf32_rn(sv - hi);
    }
    for (int q = tid; q < Ng; q += kThreads) lam[q] = G.lam[q];
    const long long my_tiles = G.ntiles > bid ? (G.ntiles - 1 - bid) / nbid + 1 : 0;
    auto load_tile = [&](long long k) {
        const Chunk tl = G.tiles[(bid + k * nbid) >> (FOLD ? 1 : 0)];
        TileInfo ti;
        ti.m_off = A.boxes[tl.box].m_off;
        ti.pp_off = A.boxes[tl.box].pp_off;
        ti.row0 = tl.start * kTN;
        ti.pad = A.boxes[tl.box].gpad;
        return ti;
    };
    for (int k = tid; k < my_tiles && k < kTileCache; k += kThreads) tinfo[k] = load_tile(k);
    auto tile_at = [&](long long k) { return k < kTileCache ? tinfo[k] : load_tile(k); };
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], kProducers);
            mbar_init(&empty[s], 1);
            mbar_init(&loaded[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 256);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 16) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const long long Ng2 = (long long)Ng * Ng;

    const long long nchunks = my_tiles * nkb;
    if (warp >= 8 && warp < 16) {
        // ---------------------------------------------------------------- converters
        // chunk h of this CTA = tile h / nkb, columns 16 (h % nkb) .. + 15, in stage h % NST.
        // Thread pt splits the 16-byte units q = pt + kProducers e (row q >> 2, unit q & 3)
        // in place: hi = tf32_rn(x) over the loaded value, lo = tf32_rn(x - hi) into the
        // other half of the stage.
        const int pt = tid - 256;
        uint32_t soff[kUnits];
#pragma unroll
        for (int e = 0; e < kUnits; ++e) {
            const int q = FOLD ? 4 * pt + e : pt + kProducers * e;   // folded: thread pt owns row pt
            soff[e] = sw64_offset(q >> 2, 4 * (q & 3));
        }
        const float sgn = parity ? -1.0f : 1.0f;
        for (long long h = 0; h < nchunks && !*abort_flag; ++h) {
            const int s = (int)(h % NST);
            unsigned char *xh = stages + (size_t)s * SB;
            unsigned char *xl = stages + (size_t)s * SB + kHalfBytes;
            if (PASS == P_ZM) {
                // transpose the [16 n][256 q] copy into the K-major operand: thread pt owns
                // row (cell) pt; consecutive threads read consecutive floats of each n row
                if (!mbar_wait(&loaded[s], (uint32_t)((h / NST) & 1), abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                const float *raw = reinterpret_cast<const float *>(stages + (size_t)s * SB + 2 * kHalfBytes);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    float x[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) x[t] = raw[(4 * u + t) * kTN + pt];
                    const float4 hv = make_float4(tf32_rn(x[0]), tf32_rn(x[1]), tf32_rn(x[2]), tf32_rn(x[3]));
                    const uint32_t off = sw64_offset(pt, 4 * u);
                    *reinterpret_cast<float4 *>(xh + off) = hv;
                    *reinterpret_cast<float4 *>(xl + off) = make_float4(
                        tf32_rn(x[0] - hv.x), tf32_rn(x[1] - hv.y), tf32_rn(x[2] - hv.z), tf32_rn(x[3] - hv.w));
                }
                fence_proxy_async();
                mbar_arrive(&full[s]);
                continue;
            }
            if (G.ragged) {
                // the stage is free once the MMA has consumed the chunk before in it; then
                // element (r, k) of the chunk (row r of the tile, column 16 cc + k) is read
                // by thread idx % 256 of idx = 16 r + k (a half warp reads 64 contiguous
                // bytes), split and stored in both halves (folded: x + sgn x_mirror first)
                if (!mbar_wait(&empty[s], (uint32_t)(((h / NST) & 1) ^ 1), abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                const TileInfo ti = tile_at(h / nkb);
                const int cc = (int)(h % nkb);
                const float *src = A.in + ti.m_off + (long long)ti.row0 * Ng;
                const int nrows = (int)min((long long)kTN, Ng2 - ti.row0);
                if (cc == 0 && pt == 0 && h / nkb + 1 < my_tiles) {
                    // the next tile's rows are one contiguous block: start bringing it into L2
                    const TileInfo tn = tile_at(h / nkb + 1);
                    const long long rows = min((long long)kTN, Ng2 - tn.row0);
                    const uint32_t bytes = (uint32_t)(rows * Ng * sizeof(float)) & ~15u;
                    if (bytes) prefetch_l2(A.in + tn.m_off + (long long)tn.row0 * Ng, bytes);
                }
                float v[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int idx = pt + kProducers * i;
                    const int r = idx >> 4, col = cc * kKB + (idx & 15);
                    float x = 0.0f;
                    if (r < nrows) {
                        const float *row = src + (long long)r * Ng;
                        if (col < Ng) x = row[col];
                        if (FOLD && Ng - 1 - col >= 0) x = fmaf(sgn, row[Ng - 1 - col], x);
                    }
                    v[i] = x;
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int idx = pt + kProducers * i;
                    const uint32_t off = sw64_offset(idx >> 4, idx & 15);
                    const float hi = tf32_rn(v[i]);
                    *(float *)(xh + off) = hi;
                    *(float *)(xl + off) = tf32_rn(v[i] - hi);
                }
                fence_proxy_async();
                mbar_arrive(&full[s]);
                continue;
            }
            if (!mbar_wait(&loaded[s], (uint32_t)((h / NST) & 1), abort_flag)) {
                *abort_flag = 1;
                break;
            }
            if (FOLD) {
                // half 0 holds columns n of the chunk, half 1 the mirror chunk (column 15 - k
                // there pairs with column k here); the row becomes w = x + sgn x_mirror, split
                // into hi (half 0) and lo (half 1) in place.  Units e and 3 - e of each half
                // hold mirror columns: take them in pairs
#pragma unroll
                for (int e = 0; e < kUnits / 2; ++e) {
                    const float4 c0 = *reinterpret_cast<const float4 *>(xh + soff[e]);
                    const float4 c1 = *reinterpret_cast<const float4 *>(xh + soff[3 - e]);
                    const float4 m0 = *reinterpret_cast<const float4 *>(xl + soff[e]);
                    const float4 m1 = *reinterpret_cast<const float4 *>(xl + soff[3 - e]);
                    // column 4e + j pairs with mirror column 15 - 4e - j = 4 (3 - e) + (3 - j)
                    const float4 w0 = make_float4(fmaf(sgn, m1.w, c0.x), fmaf(sgn, m1.z, c0.y),
                                                  fmaf(sgn, m1.y, c0.z), fmaf(sgn, m1.x, c0.w));
                    const float4 w1 = make_float4(fmaf(sgn, m0.w, c1.x), fmaf(sgn, m0.z, c1.y),
                                                  fmaf(sgn, m0.y, c1.z), fmaf(sgn, m0.x, c1.w));
                    const float4 h0 = make_float4(tf32_rn(w0.x), tf32_rn(w0.y), tf32_rn(w0.z), tf32_rn(w0.w));
                    const float4 h1 = make_float4(tf32_rn(w1.x), tf32_rn(w1.y), tf32_rn(w1.z), tf32_rn(w1.w));
                    *reinterpret_cast<float4 *>(xh + soff[e]) = h0;
                    *reinterpret_cast<float4 *>(xh + soff[3 - e]) = h1;
                    *reinterpret_cast<float4 *>(xl + soff[e]) = make_float4(
                        tf32_rn(w0.x - h0.x), tf32_rn(w0.y - h0.y), tf32_rn(w0.z - h0.z), tf32_rn(w0.w - h0.w));
                    *reinterpret_cast<float4 *>(xl + soff[3 - e]) = make_float4(
                        tf32_rn(w1.x - h1.x), tf32_rn(w1.y - h1.y), tf32_rn(w1.z - h1.z), tf32_rn(w1.w - h1.w));
                }
            } else {
#pragma unroll
                for (int e = 0; e < kUnits; ++e) {
                    const float4 v = *reinterpret_cast<const float4 *>(xh + soff[e]);
                    const float4 h = make_float4(tf32_rn(v.x), tf32_rn(v.y), tf32_rn(v.z), tf32_rn(v.w));
                    *reinterpret_cast<float4 *>(xh + soff[e]) = h;
                    *reinterpret_cast<float4 *>(xl + soff[e]) = make_float4(
                        tf32_rn(v.x - h.x), tf32_rn(v.y - h.y), tf32_rn(v.z - h.z), tf32_rn(v.w - h.w));
                }
            }
            fence_proxy_async();
            mbar_arrive(&full[s]);
        }
    } else if (warp == 17) {
        // ---------------------------------------------------------------- tensor copies
        // lane 0 loads chunk g into stage g % NST as soon as the MMA has released it; on an
        // abort it waits (bounded) for the copies it issued before the CTA may exit.  Idle on
        // the ragged path (the converters load the chunks themselves)
        if (lane == 0 && !G.ragged) {
            long long g = 0;
            for (; g < nchunks && !*abort_flag; ++g) {
                const int s = (int)(g % NST);
                if (!mbar_wait(&empty[s], (uint32_t)(((g / NST) & 1) ^ 1), abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                const TileInfo ti = tile_at(g / nkb);
                if (PASS == P_ZM) {
                    // planes 16 cc .. 16 cc + 15 of the box, cells row0 .. row0 + 255
                    const int cc = (int)(g % nkb), y = (int)(ti.m_off / Ng2 + cc * kKB);
                    mbar_arrive_expect_tx(&loaded[s], kHalfBytes);
                    tma_load_2d(smem_u32(stages + (size_t)s * SB + 2 * kHalfBytes), &G.in_map, ti.row0, y, &loaded[s]);
                    continue;
                }
                if (g % nkb == 0 && g / nkb + 1 < my_tiles) {
                    // the next tile's rows are one contiguous block: start bringing it into L2
                    const TileInfo tn = tile_at(g / nkb + 1);
                    const long long rows = min((long long)kTN, Ng2 - tn.row0);
                    prefetch_l2(A.in + tn.m_off + (long long)tn.row0 * Ng, (uint32_t)(rows * Ng * sizeof(float)));
                }
                const int cc = (int)(g % nkb), y = (int)(ti.m_off / Ng + ti.row0);
                mbar_arrive_expect_tx(&loaded[s], FOLD ? 2 * kHalfBytes : kHalfBytes);
                tma_load_2d(smem_u32(stages + (size_t)s * SB), &G.in_map, cc * kKB, y, &loaded[s]);
                if (FOLD)   // the mirror chunk: columns Ng - 16 (cc + 1) .. Ng - 16 cc - 1
                    tma_load_2d(smem_u32(stages + (size_t)s * SB + kHalfBytes), &G.in_map,
                                Ng - (cc + 1) * kKB, y, &loaded[s]);
            }
            if (*abort_flag) {
                const unsigned long long t0 = now_ns();
                for (long long h = g - NST > 0 ? g - NST : 0; h < g; ++h)
                    while (!mbar_try_wait(&loaded[h % NST], (uint32_t)((h / NST) & 1)) && now_ns() - t0 < kWaitNs) {
                    }
            }
        }
    } else if (warp == 16) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0 && A.stall_ns) {
            // self-test of the failure path: the drain barrier receives nothing before the
            // tear-down, so this bounded wait expires and the CTA aborts like any timeout
            const unsigned long long t0 = now_ns();
            while (!mbar_try_wait(drain, 0) && now_ns() - t0 < A.stall_ns) {
            }
            *abort_flag = 1;
        }
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(kTM, kTN);
            const uint32_t shi = smem_u32(S_hi), slo = smem_u32(S_lo), st0 = smem_u32(stages);
            long long g = 0;
            uint32_t t = 0;
            for (long long it = 0; it < my_tiles && !*abort_flag; ++it, ++t) {
                const int a = t & 1;
                if (!mbar_wait(&tempty[a], ((t >> 1) & 1) ^ 1, abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(a * kTN);
                bool ok = true;
                for (int c = 0; c < nkb; ++c, ++g) {
                    const int s = (int)(g % NST);
                    if (!mbar_wait(&full[s], (uint32_t)((g / NST) & 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t xh = st0 + (uint32_t)s * SB, xl = xh + kHalfBytes;
#pragma unroll
                    for (int kk = 0; kk < kKB / 8; ++kk) {
                        const int kg = c * kKB + kk * 8;
                        if (kg >= Nk) break;                      // all-zero K step
                        const uint32_t ao = (uint32_t)(kg / kKA) * sch + (uint32_t)((kg % kKA) / 8) * 32;
                        const uint64_t ahi = sw128_desc(shi + ao), alo = sw128_desc(slo + ao);
                        const uint64_t bhi = sw64_desc(xh + kk * 32), blo = sw64_desc(xl + kk * 32);
                        mma_tf32(d, ahi, bhi, idesc, (c | kk) != 0);
                        mma_tf32(d, ahi, blo, idesc, 1);
                        mma_tf32(d, alo, bhi, idesc, 1);
                        if (A.lo_lo) mma_tf32(d, alo, blo, idesc, 1);
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
        // warp w reads TMEM lanes 32 (w & 3) + lane (output columns n) and rows
        // 128 (w >> 2) .. + 127 of the tile, 32 at a time, and transposes each 32 x 32 block
        // through shared memory in 16-byte units, so that a 16-byte store instruction writes
        // 32 consecutive rows (128 bytes) of each of four columns.  All epilogue warps follow
        // every tile's barriers, also those whose lanes are all >= Ng.
        const int quarter = warp & 3, half = warp >> 2;
        const int n0 = quarter * 32;
        const int ncol = Nk - n0 < 32 ? Nk - n0 : 32;        // valid columns of this warp (may be <= 0)
        const float scale = (PASS == P_XI || PASS == P_ZM) ? 8.0f / ((float)(Ng + 1) * (Ng + 1) * (Ng + 1)) : 1.0f;
        // (the padded row length S depends on the box's ghost width: taken per tile below)
        float *buf = xpose + warp * (kXposeBytes / 4);
        uint32_t t = 0;
        for (long long it = 0; it < my_tiles && !*abort_flag; ++it, ++t) {
            const int a = t & 1;
            if (!mbar_wait(&tfull[a], (t >> 1) & 1, abort_flag)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const TileInfo ti = tile_at(it);
            const uint32_t tbase = tmem + (uint32_t)(a * kTN + half * 128) + ((uint32_t)n0 << 16);
            if (PASS == P_ZM) {
                // lane = output k of this warp's quarter, columns = cells q of its half tile:
                // padded Phi[i + gp][j + gp][k + gp], 32 lanes -> 32 consecutive floats.  Two
                // batches of 64 columns, each with its TMEM loads in flight together; the
                // padded offset steps by one row (S) per cell, by 2 gp rows more per mesh row
                const int gp = ti.pad;
                const int S = Ng + 2 * gp;                  // padded box < 2^31 floats
#pragma unroll 1
                for (int b64 = 0; b64 < 2; ++b64) {
                    float v[4][16];
                    if (ncol > 0) {
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) tmem_ld16_issue(tbase + (uint32_t)(b64 * 64 + cc * 16), v[cc]);
                        tmem_ld_wait();
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) tmem_regs_ready(v[cc]);
                    }
                    if (b64 == 1) {
                        tc_fence_before();
                        mbar_arrive(&tempty[a]);
                    }
                    if (ncol > 0 && lane < ncol) {
                        const int q0 = ti.row0 + half * 128 + b64 * 64;
                        int jj = q0 % Ng;
                        int off = ((q0 / Ng + gp) * S + (jj + gp)) * S;
                        float *dst = A.out + ti.pp_off + gp + n0 + lane;
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc)
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                if (q0 + cc * 16 + j < Ng2) dst[off] = v[cc][j] * scale;
                                off += S;
                                if (++jj == Ng) {
                                    jj = 0;
                                    off += 2 * gp * S;
                                }
                            }
                    }
                    __syncwarp();
                }
                continue;
            }
#pragma unroll 1
            for (int rnd = 0; rnd < 4; ++rnd) {
                float v0[16], v1[16];
                if (ncol > 0) {
                    tmem_ld16_issue(tbase + (uint32_t)(rnd * 32), v0);
                    tmem_ld16_issue(tbase + (uint32_t)(rnd * 32 + 16), v1);
                    tmem_ld_wait();
                    tmem_regs_ready(v0);
                    tmem_regs_ready(v1);
                }
                if (rnd == 3) {
                    // every column of this accumulator is in registers: release it
                    tc_fence_before();
                    mbar_arrive(&tempty[a]);
                }
                if (ncol <= 0) continue;
                // lane n -> row n of the block (its column's 32 rows), as 16-byte units
                float4 *brow = reinterpret_cast<float4 *>(buf + lane * 32);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    brow[u ^ (lane & 7)] = make_float4(v0[4 * u], v0[4 * u + 1], v0[4 * u + 2], v0[4 * u + 3]);
                    brow[(u + 4) ^ (lane & 7)] = make_float4(v1[4 * u], v1[4 * u + 1], v1[4 * u + 2], v1[4 * u + 3]);
                }
                __syncwarp();
                // this lane stores rows R .. R + 3 of columns n0 + 8 (lane >> 3) + c, c < 8:
                // eight lanes cover 32 consecutive rows (128 bytes) of one column
                const int ru = lane & 7, cg = lane >> 3;
                const long long R = (long long)ti.row0 + half * 128 + rnd * 32 + 4 * ru;
                if (G.ragged && R < Ng2) {
                    // element by element: rows R .. R + 3 may cross a row of the mesh or the
                    // end of the box, and nothing is 16-byte aligned
#pragma unroll 1
                    for (int c = 0; c < 8; ++c) {
                        const int nl = cg * 8 + c;
                        if (nl >= ncol) break;
                        const int nout = FOLD ? 2 * (n0 + nl) + parity : n0 + nl;
                        const float4 x4 = reinterpret_cast<const float4 *>(buf + nl * 32)[ru ^ (nl & 7)];
                        const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const long long row = R + e;
                            if (row >= Ng2) break;
                            const int rhi = (int)(row / Ng), rlo = (int)(row - (long long)rhi * Ng);
                            if (PASS == P_XI) {
                                const int G = ti.pad;
                                const long long S = Ng + 2 * G;
                                A.out[ti.pp_off + ((long long)(nout + G) * S + (rhi + G)) * S + (rlo + G)] = xv[e] * scale;
                            } else {
                                float y = xv[e];
                                if (PASS == P_XF) y = __fdividef(y, lam[nout] + lam[rhi] + lam[rlo]);
                                A.out[ti.m_off + (long long)nout * Ng2 + row] = y;
                            }
                        }
                    }
                } else if (R < Ng2) {
                    const int rhi = (int)(R / Ng), rlo = (int)(R - (long long)(R / Ng) * Ng);
                    float4 lr;
                    if (PASS == P_XF)
                        lr = make_float4(lam[rhi] + lam[rlo], lam[rhi] + lam[rlo + 1], lam[rhi] + lam[rlo + 2],
                                         lam[rhi] + lam[rlo + 3]);
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const int nl = cg * 8 + c;
                        if (nl >= ncol) break;
                        const int nout = FOLD ? 2 * (n0 + nl) + parity : n0 + nl;   // output column
                        float4 x = reinterpret_cast<const float4 *>(buf + nl * 32)[ru ^ (nl & 7)];
                        if (PASS == P_XI) {
                            // rows R .. R + 3 share rhi (Ng % 4 == 0); padded boxes start so that
                            // their interior rows are 16-byte aligned (pp_off + G = 0 mod 4)
                            const int G = ti.pad;
                            const long long S = Ng + 2 * G;
                            float *p = A.out + ti.pp_off + ((long long)(nout + G) * S + (rhi + G)) * S + (rlo + G);
                            *reinterpret_cast<float4 *>(p) = make_float4(x.x * scale, x.y * scale, x.z * scale, x.w * scale);
                        } else {
                            if (PASS == P_XF) {
                                const float ln = lam[nout];
                                x = make_float4(__fdividef(x.x, ln + lr.x), __fdividef(x.y, ln + lr.y),
                                                __fdividef(x.z, ln + lr.z), __fdividef(x.w, ln + lr.w));
                            }
                            *reinterpret_cast<float4 *>(A.out + ti.m_off + (long long)nout * Ng2 + R) = x;
                        }
                    }
                }
                __syncwarp();
            }
        }
    }

    // ---- tear-down: every role has left its loop; drain, then free tensor memory
    if (warp == 16 && lane == 0 && *abort_flag) {
        // wait (bounded) until every MMA this thread issued has finished writing TMEM
        mma_commit(drain);
        const unsigned long long t0 = now_ns();
        while (!mbar_try_wait(drain, 0) && now_ns() - t0 < kWaitNs) {
        }
    }
    if (*abort_flag && tid == 0) atomicOr(A.err, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 16) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// Dynamic shared memory of a launch: Nk matrix rows (Ng, or Ng / 2 folded), Ng eigenvalues.
size_t tc_smem_bytes(int Nk, int Ng, int nkc, int nstage, bool zm = false) {
    const size_t sch = (size_t)((Nk + 7) / 8) * 1024;
    return 1024 + 2 * (size_t)nkc * sch + (size_t)nstage * stage_bytes(zm ? P_ZM : P_F) + (zm ? 0 : 8 * kXposeBytes) +
           (3 * nstage + 5) * 8 + 16 +
           (size_t)Ng * 4 + 16 + kTileCache * sizeof(TileInfo) + 64;
}

constexpr size_t kSmemBudget = 227 * 1024;

// The input buffer as a 2D tensor of rows of Ng floats (box m_off are multiples of Ng), for
// 16 x 256 tensor copies with the 64-byte swizzle of the MMA stages; encoded once per
// (buffer, Ng) through the CUDA driver API's entry point (cuTensorMapEncodeTiled).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

cudaError_t input_map(Ctx &c, const float *buf, int Ng, CUtensorMap *out, bool plane_major = false) {
    static std::mutex mu;
    static std::map<std::pair<std::pair<const void *, long long>, int>, CUtensorMap> cache;
    if (plane_major) Ng = -Ng;                       // (its own cache entries)
    static EncodeTiledFn encode = nullptr;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(std::make_pair((const void *)buf, c.M), Ng);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return e != cudaSuccess ? e : cudaErrorNotSupported;
        encode = (EncodeTiledFn)fn;
    }
    CUtensorMap m;
    const cuuint32_t estr[2] = {1, 1};
    if (plane_major) {
        // rows of Ng^2 floats (one plane of a box mesh, box offsets multiples of Ng^2), boxes of
        // 256 cells x 16 planes, unswizzled (the converters transpose them)
        const long long n2 = (long long)Ng * Ng;
        const cuuint64_t dims[2] = {(cuuint64_t)n2, (cuuint64_t)(c.M / n2)};
        const cuuint64_t strides[1] = {(cuuint64_t)n2 * sizeof(float)};
        const cuuint32_t box[2] = {(cuuint32_t)kTN, (cuuint32_t)kKB};
        if (encode(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(buf), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    } else {
        const cuuint64_t dims[2] = {(cuuint64_t)Ng, (cuuint64_t)(c.M / Ng)};
        const cuuint64_t strides[1] = {(cuuint64_t)Ng * sizeof(float)};
        const cuuint32_t box[2] = {(cuuint32_t)kKB, (cuuint32_t)kTN};
        if (encode(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(buf), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    cache[key] = m;
    *out = m;
    return cudaSuccess;
}

// One launch of pass PASS over up to kMaxTcGroups Ng groups of the same form (all direct or
// all folded).  The persistent grid (one CTA per SM) is split among the groups in proportion
// to their work (items x Ng, the contraction length), each group getting at least one CTA
// (two when folded, one per parity) and no more CTAs than items.
template <int PASS>
cudaError_t run_tc_pass(Ctx &c, const std::vector<TcGroup> &groups, const float *in, float *out) {
    TcArgs a;
    std::memset(&a, 0, sizeof(a));
    const int ng = (int)groups.size();
    if (ng < 1 || ng > kMaxTcGroups) return cudaErrorInvalidValue;
    const bool fold = tc_folded(groups[0].Ng);
    const int step = fold ? 2 : 1;
    double total = 0;
    std::vector<double> work(ng);
    std::vector<int> items(ng), ctas(ng);
    for (int g = 0; g < ng; ++g) {
        items[g] = fold ? 2 * groups[g].ntiles : groups[g].ntiles;
        work[g] = (double)items[g] * groups[g].Ng;
        total += work[g];
    }
    int sum = 0;
    for (int g = 0; g < ng; ++g) {
        int n = (int)(c.num_sms * work[g] / std::max(total, 1.0)) / step * step;
        n = std::max(step, std::min(n, (items[g] + step - 1) / step * step));
        ctas[g] = n;
        sum += n;
    }
    while (sum > std::max(c.num_sms, step * ng)) {            // trim the largest share
        int g = (int)(std::max_element(ctas.begin(), ctas.end()) - ctas.begin());
        if (ctas[g] <= step) break;
        ctas[g] -= step;
        sum -= step;
    }
    size_t smem = 0;
    int cta0 = 0;
    for (int g = 0; g < ng; ++g) {
        const TcGroup &G = groups[g];
        TcGroupArgs &A = a.grp[g];
        A.ragged = (PASS != P_ZM && tc_ragged(G.Ng)) ? 1 : 0;
        if (!A.ragged) {
            cudaError_t me = input_map(c, in, G.Ng, &A.in_map, PASS == P_ZM);
            if (me != cudaSuccess) return me;
        }
        A.tiles = G.tiles;
        A.ntiles = items[g];
        A.Ng = G.Ng;
        A.Npad = G.Npad;
        A.nkc = G.nkc;
        A.nstage = PASS == P_ZM ? G.nstage_zm : G.nstage;
        A.S = c.table_arena + G.s_off;
        A.lam = c.table_arena + G.lam_off;
        A.cta0 = cta0;
        A.nctas = ctas[g];
        cta0 += ctas[g];
        smem = std::max(smem, tc_smem_bytes(fold ? (G.Ng + 1) / 2 : G.Ng, G.Ng, G.nkc, A.nstage, PASS == P_ZM));
    }
    a.ngroups = ng;
    a.boxes = c.boxes;
    a.in = in;
    a.out = out;
    a.err = c.dev_err;
    a.lo_lo = c.tc_lo_lo ? 1 : 0;
    a.stall_ns = c.tc_stall_ns;
    if (fold) k_dst_tc<PASS, true><<<cta0, kThreads, smem, c.stream>>>(a);
    else k_dst_tc<PASS, false><<<cta0, kThreads, smem, c.stream>>>(a);
    ++c.launches;
    return cudaGetLastError();
}

}  // namespace

bool tc_folded(int Ng) { return Ng > kTM; }

bool tc_ragged(int Ng) { return tc_folded(Ng) ? Ng % 32 != 0 : Ng % 4 != 0; }

int tc_plan_stages(int Ng, int &Npad, int &nkc, bool zm) {
    // as many data stages (up to 4) as fit next to the resident sine matrix, at least 2
    const int Nk = tc_folded(Ng) ? (Ng + 1) / 2 : Ng;
    Npad = ((Nk + 15) / 16) * 16;
    nkc = (Nk + kKA - 1) / kKA;
    for (int nst = 4; nst >= 2; --nst)
        if (tc_smem_bytes(Nk, Ng, nkc, nst, zm) <= kSmemBudget) return nst;
    return 0;
}

bool tc_supported(int Ng) {
    int Npad, nkc;
    // direct form: Ng <= 128 (one M = 128 operand); folded form: ceil(Ng / 2) <= 128
    return Ng >= 2 && Ng <= 2 * kTM && tc_plan_stages(Ng, Npad, nkc, false) >= 2;
}

template <int PASS>
cudaError_t set_tc_attr() {
    const int lim = (int)kSmemBudget;
    cudaError_t e = cudaFuncSetAttribute(k_dst_tc<PASS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_dst_tc<PASS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

cudaError_t init_tc_kernels() {
    cudaError_t e;
    if ((e = set_tc_attr<P_F>())) return e;
    if ((e = set_tc_attr<P_XF>())) return e;
    if ((e = set_tc_attr<P_ZI>())) return e;
    if ((e = set_tc_attr<P_YI>())) return e;
    if ((e = set_tc_attr<P_ZM>())) return e;
    if ((e = init_plane_kernel())) return e;
    return set_tc_attr<P_XI>();
}

// The launch groups: every Ng group with boxes in the bound batch, or in the per-tile form
// only the current box's tiles.
std::vector<TcGroup> active_groups(const Ctx &c) {
    std::vector<TcGroup> one;
    if (c.view_box < 0) {
        for (const TcGroup &G : c.tc_groups)
            if (G.ntiles > 0) one.push_back(G);       // (a batch may hold no box of an Ng)
        return one;
    }
    for (const TcGroup &G : c.tc_groups) {
        if (G.Ng != c.boxes_h[c.view_box].Ng) continue;
        TcGroup V = G;
        V.tiles = c.tc_tiles + c.tc_tile_beg[c.view_box];
        V.ntiles = c.tc_tile_end[c.view_box] - c.tc_tile_beg[c.view_box];
        if (c.tc_planes) {
            V.planes = c.tc_planes + c.tc_plane_beg[c.view_box];
            V.nplanes = G.Ng;
        }
        one.push_back(V);
    }
    return one;
}

// The active groups split into launches: direct and folded forms apart, at most kMaxTcGroups
// groups each (every workload here makes one launch per pass).
std::vector<std::vector<TcGroup>> tc_launches(const Ctx &c) {
    std::vector<std::vector<TcGroup>> out;
    for (int f = 0; f < 2; ++f) {
        std::vector<TcGroup> cur;
        for (const TcGroup &G : active_groups(c)) {
            if ((int)tc_folded(G.Ng) != f) continue;
            cur.push_back(G);
            if ((int)cur.size() == kMaxTcGroups) {
                out.push_back(cur);
                cur.clear();
            }
        }
        if (!cur.empty()) out.push_back(cur);
    }
    return out;
}

cudaError_t launch_poisson_tc_pass(Ctx &c, int pass) {
    if (c.tc3) {
        // three passes: source (work2) -> work (z+) -> work2 (plane) -> phi (z-)
        if (pass >= 3) return cudaSuccess;
        cudaError_t e = cudaSuccess;
        for (const auto &L : tc_launches(c)) {
            if (pass == 0) e = run_tc_pass<P_F>(c, L, c.work2, c.work);
            else if (pass == 1) e = launch_plane_pass(c, L, c.work, c.work2);
            else e = run_tc_pass<P_ZM>(c, L, c.work2, c.phi);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    // buffers: source (work2) -> work -> work2 -> work -> work2 -> work -> phi
    cudaError_t e = cudaSuccess;
    for (const auto &L : tc_launches(c)) {
        switch (pass) {
            case 0: e = run_tc_pass<P_F>(c, L, c.work2, c.work); break;
            case 1: e = run_tc_pass<P_F>(c, L, c.work, c.work2); break;
            case 2: e = run_tc_pass<P_XF>(c, L, c.work2, c.work); break;
            case 3: e = run_tc_pass<P_ZI>(c, L, c.work, c.work2); break;
            case 4: e = run_tc_pass<P_YI>(c, L, c.work2, c.work); break;
            case 5: e = run_tc_pass<P_XI>(c, L, c.work, c.phi); break;
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
    if (c.tc3) {
        for (const auto &L : tc_launches(c)) {
            e = run_tc_pass<P_F>(c, L, in, w1);
            if (e == cudaSuccess) e = launch_plane_pass(c, L, w1, w2);
            if (e == cudaSuccess) e = run_tc_pass<P_ZM>(c, L, w2, out_pad);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    for (const auto &L : tc_launches(c)) {
        e = run_tc_pass<P_F>(c, L, in, w1);
        if (e == cudaSuccess) e = run_tc_pass<P_F>(c, L, w1, w2);
        if (e == cudaSuccess) e = run_tc_pass<P_XF>(c, L, w2, w1);
        if (e == cudaSuccess) e = run_tc_pass<P_ZI>(c, L, w1, w2);
        if (e == cudaSuccess) e = run_tc_pass<P_YI>(c, L, w2, w1);
        if (e == cudaSuccess) e = run_tc_pass<P_XI>(c, L, w1, out_pad);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace scola
