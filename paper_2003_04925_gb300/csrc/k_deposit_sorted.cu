// CIC deposit B^sCOLA (Sec. 3.4.1) and the Poisson source delta' = delta - Lap Phi_BC
// (App. C, Eq. 62) by sorting the particles by brick and reducing in shared memory.
//
// The interior mesh of a box is cut into bricks of 16^3 cells; brick b owns cells
// [16 b, 16 b + 16) along each axis.  A particle whose clamped mesh coordinate has integer
// part i0 puts CIC weight on cells i0 and i0 + 1 along each axis.  It is keyed by the
// brick that owns its upper corner, ((i0 + 1) >> 4) per axis, and by a 3-bit class whose
// bit a says that its lower corner lies in the brick below along axis a ((i0_a + 1) is a
// multiple of 16).  The key grid has one extra brick per axis (index nb = ceil(Ng / 16))
// for particles whose upper corner is just outside the mesh.  Particles with no corner
// inside the mesh are dropped (their weight is outside, as B^sCOLA requires).
//
//   count  per-key entry counts (one warp-aggregated atomic per distinct key in a warp)
//   scan   per-box exclusive prefix sums of the counts: each key's slice of the box's list
//   fill   every particle writes (f_x, f_y, f_z, packed i0) into its key's slice
//   brick  one CTA per real brick reads its own 8 class slices and the slices of its 7
//          upper neighbours whose class bits point back at it (about 1.2 entries per
//          particle), adds the CIC weights that fall in its cells to 2^-32 fixed-point
//          counters in shared memory, then writes delta and delta' for its cells.
// Integer sums do not depend on the order of the additions, so the result is the same
// for any order of the entries within a slice.
#include "device_util.cuh"

namespace scola {

namespace {

constexpr int kBrickCells = kBrick * kBrick * kBrick;

// The (neighbour offset d, class c) pairs with (c & d) == d: the slices a brick reads.
constexpr int kSegments = 27;
__constant__ int kSegD[kSegments] = {0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 4, 4, 4, 4, 5, 5, 6, 6, 7};
__constant__ int kSegC[kSegments] = {0, 1, 2, 3, 4, 5, 6, 7, 1, 3, 5, 7, 2, 3, 6, 7, 3, 7, 4, 5, 6, 7, 5, 7, 6, 7, 7};

__device__ __forceinline__ SortEntry sort_entry(const BoxDesc &B, const float *__restrict__ s, long long stride,
                                                int local) {
    int b[3];
    decode_local(local, B.Nsc, b[0], b[1], b[2]);
    const long long gi = B.p_off + local;
    const float sv[3] = {__ldg(s + gi), __ldg(s + stride + gi), __ldg(s + 2 * stride + gi)};
    return brick_entry(B, sv, b);
}

// FILL = false: add each key's entries of this chunk to the counts.  FILL = true: reserve
// slots through the cursors and write the entries.  One atomic per distinct key per warp.
// A reservation past the slots the count pass gave a key (offs + cnt) would mean that the
// two passes disagreed on a key: it is recorded in err (bit 2) and nothing is written.
template <bool FILL>
__global__ void __launch_bounds__(kChunk)
k_sort_bin(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks, int nchunks, const float *__restrict__ s,
           long long stride, int *__restrict__ ctr, float4 *__restrict__ entries, const int *__restrict__ cnt,
           const int *__restrict__ offs, int *__restrict__ err) {
    // two chunks per CTA: both particles' loads, and then both reservations, are in flight
    // together
    SortEntry se[2];
    int kb[2];
    long long pb[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        se[u].key = -1;
        kb[u] = 0;
        pb[u] = 0;
        const int ci = 2 * blockIdx.x + u;
        if (ci < nchunks) {
            const Chunk ch = chunks[ci];
            const BoxDesc &B = boxes[ch.box];
            kb[u] = B.key_off;
            pb[u] = B.p_off;
            const int local = ch.start + threadIdx.x;
            if (local < B.Nsc * B.Nsc * B.Nsc) se[u] = sort_entry(B, s, stride, local);
        }
    }
    const int lane = threadIdx.x & 31;
    unsigned peers[2];
    int leader[2], base[2] = {0, 0}, ok[2] = {1, 1};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        peers[u] = __match_any_sync(0xffffffffu, se[u].key);   // every lane takes part
        leader[u] = __ffs(peers[u]) - 1;
    }
    if (!FILL) {
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (se[u].key >= 0 && lane == leader[u]) atomicAdd(ctr + kb[u] + se[u].key, __popc(peers[u]));
        return;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
        if (se[u].key >= 0 && lane == leader[u]) base[u] = atomicAdd(ctr + kb[u] + se[u].key, __popc(peers[u]));
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        if (se[u].key >= 0 && lane == leader[u]) {
            ok[u] = base[u] + __popc(peers[u]) <= offs[kb[u] + se[u].key] + cnt[kb[u] + se[u].key];
            if (!ok[u]) atomicOr(err, 2);
        }
        base[u] = __shfl_sync(0xffffffffu, base[u], leader[u]);
        ok[u] = __shfl_sync(0xffffffffu, ok[u], leader[u]);
        if (se[u].key >= 0 && ok[u])
            entries[pb[u] + base[u] + __popc(peers[u] & ((1u << lane) - 1u))] = se[u].e;
    }
}

// Exclusive prefix sums of one box's key counts (one CTA of 1024 threads per box).
__global__ void __launch_bounds__(1024)
k_sort_scan(const BoxDesc *__restrict__ boxes, int box0, const int *__restrict__ cnt, int *__restrict__ offs,
            int *__restrict__ cursor) {
    const BoxDesc &B = boxes[box0 + blockIdx.x];
    const int n = B.nbe * B.nbe * B.nbe * 8, off = B.key_off;
    __shared__ int wsum[32];
    __shared__ int carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 1024) {
        const int i = base + tid;
        const int v = i < n ? cnt[off + i] : 0;
        int x = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = wsum[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const int excl = carry + (warp ? wsum[warp - 1] : 0) + x - v;
        if (i < n) {
            offs[off + i] = excl;
            cursor[off + i] = excl;
        }
        __syncthreads();
        if (tid == 1023) carry = excl + v;
        __syncthreads();
    }
}

__device__ __forceinline__ void store4(float *p, const float (&v)[4], bool vec, int left) {
    if (vec) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
        return;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e)
        if (e < left) p[e] = v[e];
}

// Adds fixed-point weight f (at most 2^32) to a count kept as two 32-bit halves: a 32-bit
// add to the low half, and a carry into the high half when it wraps (the same integer sum
// as a 64-bit add, in 32-bit shared-memory atomics).
__device__ __forceinline__ void add_split(unsigned *lo, unsigned *hi, int c, unsigned long long f) {
    if (f >> 32) {                      // a weight of exactly 1
        atomicAdd(hi + c, 1u);
        return;
    }
    const unsigned v = (unsigned)f;
    const unsigned old = atomicAdd(lo + c, v);
    if (old > 0xffffffffu - v) atomicAdd(hi + c, 1u);
}

// Adds fixed-point weight f (at most 2^32) as its low 16 bits and the rest (at most 2^16) to two
// 32-bit counters with reductions that return nothing: the count is hi 2^16 + lo, exact while
// a cell receives at most 65535 weights (a brick with at most 65535 entries).
__device__ __forceinline__ void add_red16(unsigned *lo, unsigned *hi, int c, unsigned long long f) {
    atomicAdd(lo + c, (unsigned)(f & 0xffffu));
    atomicAdd(hi + c, (unsigned)(f >> 16));
}

// Counter modes of the brick pass: 64-bit atomics; 32-bit halves with a carry; 16-bit halves
// with reductions (bricks with more than 65535 entries take the carry form).
enum { kAcc64 = 0, kAccHalves = 1, kAccRed16 = 2 };

// Adds the CIC weights of one entry (fractions v.xyz, packed lower cell v.w) that fall in the
// brick [x0, x0 + 16) x [y0, ..) x [z0, ..) to its counters.  kFull: the brick lies inside
// the mesh, so only the brick bounds need checking.
template <int kMode, bool kFull>
__device__ __forceinline__ void deposit_entry(unsigned long long *acc, const float4 v, int x0, int y0, int z0,
                                              int Ng) {
    const int pk = __float_as_int(v.w);
    const int lx = (pk & 1023) - 2 - x0, ly = ((pk >> 10) & 1023) - 2 - y0, lz = ((pk >> 20) & 1023) - 2 - z0;
#pragma unroll
    for (int ex = 0; ex < 2; ++ex) {
        const int cx = lx + ex;
        if ((unsigned)cx >= (unsigned)kBrick || (!kFull && x0 + cx >= Ng)) continue;
        const float wx = ex ? v.x : 1.0f - v.x;
#pragma unroll
        for (int ey = 0; ey < 2; ++ey) {
            const int cy = ly + ey;
            if ((unsigned)cy >= (unsigned)kBrick || (!kFull && y0 + cy >= Ng)) continue;
            const float wxy = wx * (ey ? v.y : 1.0f - v.y);
#pragma unroll
            for (int ez = 0; ez < 2; ++ez) {
                const int cz = lz + ez;
                if ((unsigned)cz >= (unsigned)kBrick || (!kFull && z0 + cz >= Ng)) continue;
                const unsigned long long f = weight_to_fixed(wxy * (ez ? v.z : 1.0f - v.z));
                const int cell = (cx * kBrick + cy) * kBrick + cz;
                if (kMode == kAccHalves) {
                    unsigned *lo = reinterpret_cast<unsigned *>(acc);
                    add_split(lo, lo + kBrickCells, cell, f);
                } else if (kMode == kAccRed16) {
                    unsigned *lo = reinterpret_cast<unsigned *>(acc);
                    add_red16(lo, lo + kBrickCells, cell, f);
                } else {
                    atomicAdd(&acc[cell], f);
                }
            }
        }
    }
}

// One CTA of T threads per real brick (item.start = brick index in the box, nb^3 of them).
// kMode: the counter form (kAcc64, kAccHalves, kAccRed16).
template <int kBrickThreads, int kMode>
__global__ void __launch_bounds__(kBrickThreads, kBrickThreads == 256 ? 6 : 3)
k_sort_brick(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ items, const int *__restrict__ cnt,
             const int *__restrict__ offs, const float4 *__restrict__ entries, const float *__restrict__ phi_pad,
             float inv_D1, const float *__restrict__ coef, int kstep, int nk, float *__restrict__ out,
             float *__restrict__ delta_out) {
    __shared__ __align__(16) unsigned long long acc[kBrickCells];
    __shared__ int seg_o[kSegments], seg_start[kSegments + 1];
    const Chunk it = items[blockIdx.x];
    const BoxDesc &B = boxes[it.box];
    if (const float *cf = box_coef(coef, it.box, kstep, nk)) inv_D1 = cf[6];
    const int Ng = B.Ng, nbe = B.nbe, nb = nbe - 1;
    const int tid = threadIdx.x;
    const int bz = it.start % nb, bt = it.start / nb, by = bt % nb, bx = bt / nb;
    const int x0 = bx * kBrick, y0 = by * kBrick, z0 = bz * kBrick;
    for (int q = tid; q < kBrickCells / 2; q += kBrickThreads)
        reinterpret_cast<ulonglong2 *>(acc)[q] = make_ulonglong2(0ull, 0ull);
    const float4 *list = entries + B.p_off;
    // the 27 slices this brick reads: neighbour offset d (bit a: +1 along axis a) and class
    // c with (c & d) == d; warp 0 loads their counts and offsets and scans the counts
    if (tid < 32) {
        int n = 0;
        if (tid < kSegments) {
            const int d = kSegD[tid], c = kSegC[tid];
            const int key = B.key_off + (((bx + (d & 1)) * nbe + (by + ((d >> 1) & 1))) * nbe + (bz + (d >> 2))) * 8 + c;
            n = cnt[key];
            seg_o[tid] = offs[key];
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, n, o);
            if (tid >= o) n += y;
        }
        if (tid < kSegments) seg_start[tid + 1] = n;
        if (tid == 0) seg_start[0] = 0;
    }
    __syncthreads();
    // the brick's own 8 class slices are consecutive keys, hence one contiguous range: two
    // entries per thread and iteration (both loads in flight); then the spill slices of the
    // seven upper neighbours, located by a search over their 19 segment starts
    const int own = seg_start[8], total = seg_start[kSegments];
    const float4 *own_list = list + seg_o[0];
    const bool full = x0 + kBrick <= Ng && y0 + kBrick <= Ng && z0 + kBrick <= Ng;
    // the 16-bit form needs at most 65535 weights per cell: bricks with more entries (uniform
    // per CTA) take the carry form in the same counters
    const bool red16 = kMode == kAccRed16 && total <= 65535;
    auto deposit = [&](const float4 &v) {
        if (kMode == kAccRed16 && !red16) {
            if (full) deposit_entry<kAccHalves, true>(acc, v, x0, y0, z0, Ng);
            else deposit_entry<kAccHalves, false>(acc, v, x0, y0, z0, Ng);
        } else {
            if (full) deposit_entry<kMode, true>(acc, v, x0, y0, z0, Ng);
            else deposit_entry<kMode, false>(acc, v, x0, y0, z0, Ng);
        }
    };
    for (int e = tid; e < own; e += 2 * kBrickThreads) {
        const bool two = e + kBrickThreads < own;
        const float4 v0 = own_list[e];
        const float4 v1 = two ? own_list[e + kBrickThreads] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        deposit(v0);
        if (two) deposit(v1);
    }
    for (int e = own + tid; e < total; e += kBrickThreads) {
        int lo = 8, hi = kSegments;              // seg_start[lo] <= e < seg_start[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (seg_start[mid] <= e) lo = mid;
            else hi = mid;
        }
        deposit(list[seg_o[lo] + e - seg_start[lo]]);
    }
    __syncthreads();
    // cells: item q -> (x, y) row of the brick, 4 consecutive z cells
    const float sc = B.nbar_inv * 2.3283064365386963e-10f, c2 = B.inv_dg * B.inv_dg;
    const int G = B.gpad, ng = B.fda / 2, S = Ng + 2 * G;
    const bool edge = x0 == 0 || y0 == 0 || z0 == 0 || x0 + kBrick >= Ng || y0 + kBrick >= Ng || z0 + kBrick >= Ng;
    for (int q = tid; q < kBrickCells / 4; q += kBrickThreads) {
        const int lz = (q % (kBrick / 4)) * 4, ly = (q / (kBrick / 4)) % kBrick, lx = q / (kBrick * kBrick / 4);
        const int i = x0 + lx, j = y0 + ly, k = z0 + lz;
        if (i >= Ng || j >= Ng || k >= Ng) continue;
        ulonglong2 a01, a23;
        if (kMode != kAcc64) {
            const unsigned *lo = reinterpret_cast<const unsigned *>(acc) + (lx * kBrick + ly) * kBrick + lz;
            const uint4 l = *reinterpret_cast<const uint4 *>(lo);
            const uint4 h = *reinterpret_cast<const uint4 *>(lo + kBrickCells);
            const int sh = red16 ? 16 : 32;
            a01 = make_ulonglong2(((unsigned long long)h.x << sh) + l.x, ((unsigned long long)h.y << sh) + l.y);
            a23 = make_ulonglong2(((unsigned long long)h.z << sh) + l.z, ((unsigned long long)h.w << sh) + l.w);
        } else {
            const ulonglong2 *a = reinterpret_cast<const ulonglong2 *>(acc + (lx * kBrick + ly) * kBrick + lz);
            a01 = a[0];
            a23 = a[1];
        }
        float v[4];
        v[0] = fixed_to_float(a01.x) * sc - 1.0f;
        v[1] = fixed_to_float(a01.y) * sc - 1.0f;
        v[2] = fixed_to_float(a23.x) * sc - 1.0f;
        v[3] = fixed_to_float(a23.y) * sc - 1.0f;
        const long long cell = B.m_off + ((long long)i * Ng + j) * Ng + k;
        const bool vec = k + 4 <= Ng && (Ng & 3) == 0;
        if (delta_out) store4(delta_out + cell, v, vec, Ng - k);
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] *= inv_D1;
        if (edge && (i < ng || j < ng || i >= Ng - ng || j >= Ng - ng || k < ng || k + 4 > Ng - ng)) {
            // boundary source: the order-n Laplacian's reach into the ghost layers
            const float *Pc = phi_pad + B.pp_off + ((i + G) * S + (j + G)) * S + (k + G);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (k + e >= Ng) break;
                v[e] -= boundary_term(Pc + e, i, j, k + e, Ng, S, B.fda) * c2;
            }
        }
        store4(out + cell, v, vec, Ng - k);
    }
}

}  // namespace

// Shared memory is the brick kernel's occupancy limit: ask for the largest carveout.
cudaError_t init_deposit_kernels() {
    const void *fns[] = {(const void *)k_sort_brick<256, kAcc64>, (const void *)k_sort_brick<512, kAcc64>,
                         (const void *)k_sort_brick<256, kAccHalves>, (const void *)k_sort_brick<512, kAccHalves>,
                         (const void *)k_sort_brick<256, kAccRed16>};
    for (const void *f : fns) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                             cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Zeroes the key counts of the boxes of the current view.
cudaError_t clear_key_counts(Ctx &c) {
    const int box0 = c.view_box >= 0 ? c.view_box : 0;
    const int nbox = c.view_box >= 0 ? 1 : c.nboxes;
    const BoxDesc &first = c.boxes_h[box0];
    const BoxDesc &last = c.boxes_h[box0 + nbox - 1];
    const long long k0 = first.key_off;
    const long long nk = last.key_off + 8LL * last.nbe * last.nbe * last.nbe - k0;
    cudaError_t e = cudaMemsetAsync(c.kcount + k0, 0, sizeof(int) * (size_t)nk, c.stream);
    return e == cudaSuccess ? e : step_error("sorted deposit: clearing the key counts", e);
}

cudaError_t launch_deposit_sorted(Ctx &c, const float *s, long long stride, float inv_D1, float *delta_out,
                                  bool counted, int kstep) {
    const float *coef = kstep >= 0 ? c.coef : nullptr;
    // the boxes of the current view: all, or one in the per-tile form
    const int box0 = c.view_box >= 0 ? c.view_box : 0;
    const int nbox = c.view_box >= 0 ? 1 : c.nboxes;
    // each step's error is reported with the step's name; `counted`: the kick-drift that
    // moved these particles has already counted their keys (into cleared counts)
    cudaError_t e;
    if (!counted) {
        if ((e = clear_key_counts(c)) != cudaSuccess) return e;
        k_sort_bin<false><<<(c.n_pchunks + 1) / 2, kChunk, 0, c.stream>>>(c.boxes, c.pchunks, c.n_pchunks, s, stride,
                                                                          c.kcount, nullptr, nullptr, nullptr, nullptr);
        if ((e = cudaGetLastError()) != cudaSuccess) return step_error("sorted deposit: count launch", e);
        ++c.launches;
    }
    k_sort_scan<<<nbox, 1024, 0, c.stream>>>(c.boxes, box0, c.kcount, c.koffs, c.kcursor);
    if ((e = cudaGetLastError()) != cudaSuccess) return step_error("sorted deposit: scan launch", e);
    k_sort_bin<true><<<(c.n_pchunks + 1) / 2, kChunk, 0, c.stream>>>(c.boxes, c.pchunks, c.n_pchunks, s, stride,
                                                                     c.kcursor, c.sentries, c.kcount, c.koffs, c.dev_err);
    if ((e = cudaGetLastError()) != cudaSuccess) return step_error("sorted deposit: fill launch", e);
#define SCOLA_BRICK(T, MODE)                                                                              \
    k_sort_brick<T, MODE><<<c.n_sbricks, T, 0, c.stream>>>(c.boxes, c.sbricks, c.kcount, c.koffs, c.sentries, \
                                                           c.phi, inv_D1, coef, kstep, c.coef_nk, c.work2, delta_out)
    if (c.deposit_split == kAccRed16) SCOLA_BRICK(256, kAccRed16);
    else if (c.deposit_threads == 256) {
        if (c.deposit_split == kAccHalves) SCOLA_BRICK(256, kAccHalves);
        else SCOLA_BRICK(256, kAcc64);
    } else {
        if (c.deposit_split == kAccHalves) SCOLA_BRICK(512, kAccHalves);
        else SCOLA_BRICK(512, kAcc64);
    }
#undef SCOLA_BRICK
    if ((e = cudaGetLastError()) != cudaSuccess) return step_error("sorted deposit: brick launch", e);
    c.launches += 3;
    return cudaSuccess;
}

}  // namespace scola
