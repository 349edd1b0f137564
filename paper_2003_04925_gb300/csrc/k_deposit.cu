// CIC deposit with the mass drop B^sCOLA (Sec. 3.4.1) and the Dirichlet source of the
// Poisson solve, delta' = delta - Lap Phi_BC (App. C, Eq. 62).
//
// Every box particle adds its eight CIC weights to the interior cells they fall on, as
// 2^-32 fixed-point integers with 64-bit atomics (weight outside [0, Ng)^3 is dropped;
// the conversions to and from fixed point use 32-bit instructions only);
// integer sums do not depend on the order of the additions, so the density is
// bit-reproducible.  The counts of all boxes together would not fit in L2, so the boxes
// are taken in groups whose counts do (one scratch accumulator, reused by every group):
// for each group, the deposit kernel accumulates into the scratch, then the source kernel
// converts the counts to delta = (Ng/Nsc)^3 n - 1, subtracts the boundary term on the
// faces and writes delta' to the interior mesh, and the scratch is cleared.  The
// accumulator traffic stays in L2; HBM sees the positions once and delta' once.
#include <algorithm>

#include "device_util.cuh"

namespace scola {

namespace {

// Consecutive lanes hold Lagrangian neighbours along z (k fastest).  Where a lane's lower
// CIC corner is its left neighbour's lower corner moved one cell up in z (the common case on
// meshes of one cell per particle spacing), the neighbour's four upper-z weights fall on this
// lane's four lower-z cells: the lane adds them to its own (integer sums: the same totals)
// and the neighbour skips those atomics.
__global__ void __launch_bounds__(kChunk)
k_deposit(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks, const float *__restrict__ s,
          long long stride, unsigned long long *__restrict__ acc, long long acc_base) {
    const Chunk ch = chunks[blockIdx.x];
    const BoxDesc &B = boxes[ch.box];
    const int Nsc = B.Nsc, Ng = B.Ng;
    const int local = ch.start + threadIdx.x;
    const bool valid = local < Nsc * Nsc * Nsc;       // (every lane takes part in the shuffles)
    int i0[3] = {-1000, -1000, -1000};
    float f[3] = {0.f, 0.f, 0.f};
    if (valid) {
        const long long gi = B.p_off + local;
        int b[3];
        decode_local(local, Nsc, b[0], b[1], b[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float u = fmaf(__ldg(s + a * stride + gi), B.inv_dg, fmaf((float)b[a], B.q2u, 0.5f * B.q2u - 0.5f));
            u = fminf(fmaxf(u, -2.0f), (float)Ng + 1.0f);
            const float fl = floorf(u);
            i0[a] = (int)fl;
            f[a] = u - fl;
        }
    }
    // fixed-point weights of the eight corners
    unsigned long long w[2][2][2];
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
        const float wx = dx ? f[0] : 1.0f - f[0];
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const float wxy = wx * (dy ? f[1] : 1.0f - f[1]);
#pragma unroll
            for (int dz = 0; dz < 2; ++dz) w[dx][dy][dz] = valid ? weight_to_fixed(wxy * (dz ? f[2] : 1.0f - f[2])) : 0ull;
        }
    }
    const int lane = threadIdx.x & 31;
    const int px = __shfl_up_sync(0xffffffffu, i0[0], 1), py = __shfl_up_sync(0xffffffffu, i0[1], 1),
              pz = __shfl_up_sync(0xffffffffu, i0[2], 1);
    const bool take = valid && lane > 0 && px == i0[0] && py == i0[1] && pz + 1 == i0[2];
    const bool give = __shfl_down_sync(0xffffffffu, take ? 1 : 0, 1) && lane < 31;
#pragma unroll
    for (int dx = 0; dx < 2; ++dx)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const unsigned long long up = __shfl_up_sync(0xffffffffu, w[dx][dy][1], 1);
            if (take) w[dx][dy][0] += up;
        }
    if (!valid) return;
    unsigned long long *base = acc + (B.m_off - acc_base);
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
        const int cx = i0[0] + dx;
        if ((unsigned)cx >= (unsigned)Ng) continue;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const int cy = i0[1] + dy;
            if ((unsigned)cy >= (unsigned)Ng) continue;
#pragma unroll
            for (int dz = 0; dz < 2; ++dz) {
                const int cz = i0[2] + dz;
                if ((unsigned)cz >= (unsigned)Ng || (dz == 1 && give)) continue;
                atomicAdd(base + ((long long)cx * Ng + cy) * Ng + cz, w[dx][dy][dz]);
            }
        }
    }
}

// Four consecutive cells (a float4 where aligned), or the first `left` of them.
__device__ __forceinline__ void store4(float *p, const float (&v)[4], bool vec, int left) {
    if (vec) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
        return;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e)
        if (e < left) p[e] = v[e];
}

// Counts -> delta (optional copy) -> delta' for 4 consecutive cells per thread; a CTA takes
// kSourceChunks consecutive 256-cell chunks of the list (64 threads each).
constexpr int kSourceChunks = 4;

__global__ void __launch_bounds__(64 * kSourceChunks)
k_density_source(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks, int nchunks,
                 const unsigned long long *__restrict__ acc, long long acc_base, const float *__restrict__ phi_pad,
                 float inv_D1, const float *__restrict__ coef, int kstep, int nk, float *__restrict__ out,
                 float *__restrict__ delta_out) {
    const int ci = blockIdx.x * kSourceChunks + (threadIdx.x >> 6);
    if (ci >= nchunks) return;
    const Chunk ch = chunks[ci];
    const BoxDesc &B = boxes[ch.box];
    if (const float *cf = box_coef(coef, ch.box, kstep, nk)) inv_D1 = cf[6];
    const int Ng = B.Ng;
    const long long ng3 = (long long)Ng * Ng * Ng;
    const int cell0 = ch.start + 4 * (threadIdx.x & 63);
    if ((long long)cell0 >= ng3) return;
    const int left = (int)min(4LL, ng3 - cell0);
    const float sc = B.nbar_inv * 2.3283064365386963e-10f, c2 = B.inv_dg * B.inv_dg;
    const unsigned long long *a = acc + (B.m_off - acc_base) + cell0;
    const bool vec = left == 4 && (Ng & 3) == 0;
    float v[4];
    if (vec) {
        const ulonglong2 a01 = *reinterpret_cast<const ulonglong2 *>(a);
        const ulonglong2 a23 = *reinterpret_cast<const ulonglong2 *>(a + 2);
        v[0] = fixed_to_float(a01.x) * sc - 1.0f;
        v[1] = fixed_to_float(a01.y) * sc - 1.0f;
        v[2] = fixed_to_float(a23.x) * sc - 1.0f;
        v[3] = fixed_to_float(a23.y) * sc - 1.0f;
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            v[e] = 0.0f;
            if (e < left) v[e] = fixed_to_float(a[e]) * sc - 1.0f;
        }
    }
    const long long cell = B.m_off + cell0;
    if (delta_out) store4(delta_out + cell, v, vec, left);
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] *= inv_D1;
    // boundary source: the order-n Laplacian's reach into the ghost layers (Dirichlet values,
    // the unscaled shell) from the cells within N_ghost of a face
    int k = cell0 % Ng, j = (cell0 / Ng) % Ng, i = cell0 / Ng / Ng;
    const int G = B.gpad, ng = B.fda / 2, S = Ng + 2 * G;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (e >= left) break;
        if (k == Ng) {                          // the 4 cells cross a row (Ng % 4 != 0)
            k = 0;
            if (++j == Ng) {
                j = 0;
                ++i;
            }
        }
        if (i < ng || j < ng || k < ng || i >= Ng - ng || j >= Ng - ng || k >= Ng - ng) {
            const float *P = phi_pad + B.pp_off + ((i + G) * S + (j + G)) * S + (k + G);
            v[e] -= boundary_term(P, i, j, k, Ng, S, B.fda) * c2;
        }
        ++k;
    }
    store4(out + cell, v, vec, left);
}

}  // namespace

cudaError_t launch_deposit_atomic(Ctx &c, const float *s, long long stride, float inv_D1, float *delta_out,
                                  int kstep) {
    const float *coef = kstep >= 0 ? c.coef : nullptr;
    // box groups of the current view: the precomputed groups, or the one box of the
    // per-tile form (whose lists the view has already restricted)
    const bool one = c.view_box >= 0;
    const int ngroups = one ? 1 : (int)c.dep_groups.size() - 1;
    for (int g = 0; g < ngroups; ++g) {
        const int b0 = one ? c.view_box : c.dep_groups[g];
        const int b1 = one ? c.view_box + 1 : c.dep_groups[g + 1];
        const Chunk *pch = one ? c.pchunks : c.pchunks + c.pbeg[b0];
        const int npch = one ? c.n_pchunks : c.pbeg[b1] - c.pbeg[b0];
        const Chunk *mch = one ? c.mchunks : c.mchunks + c.mbeg[b0];
        const int nmch = one ? c.n_mchunks : c.mbeg[b1] - c.mbeg[b0];
        const long long base = c.boxes_h[b0].m_off;
        cudaError_t e;
        if (npch > 0) {
            k_deposit<<<npch, kChunk, 0, c.stream>>>(c.boxes, pch, s, stride, c.dep_acc, base);
            ++c.launches;
            if ((e = cudaGetLastError()) != cudaSuccess) return step_error("atomic deposit: deposit launch", e);
        }
        if (nmch > 0) {
            k_density_source<<<(nmch + kSourceChunks - 1) / kSourceChunks, 64 * kSourceChunks, 0, c.stream>>>(
                c.boxes, mch, nmch, c.dep_acc, base, c.phi, inv_D1, coef, kstep, c.coef_nk, c.work2, delta_out);
            ++c.launches;
            if ((e = cudaGetLastError()) != cudaSuccess) return step_error("atomic deposit: source launch", e);
        }
        // clear the counts this group used (they stay in L2 for the next group)
        const BoxDesc &last = c.boxes_h[b1 - 1];
        const long long used = last.m_off + (long long)last.Ng * last.Ng * last.Ng - base;
        e = cudaMemsetAsync(c.dep_acc, 0, sizeof(unsigned long long) * (size_t)used, c.stream);
        if (e != cudaSuccess) return step_error("atomic deposit: clearing the scratch", e);
    }
    return cudaSuccess;
}

// The deposit in the form the context selected (both give bit-identical delta').
cudaError_t launch_deposit(Ctx &c, const float *s, long long stride, float inv_D1, float *delta_out,
                           bool counted, int k) {
    return c.deposit_form == 0 ? launch_deposit_sorted(c, s, stride, inv_D1, delta_out, counted, k)
                               : launch_deposit_atomic(c, s, stride, inv_D1, delta_out, k);
}

}  // namespace scola
