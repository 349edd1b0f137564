// Per-box particle-mesh step of sCOLA (Sec. 3.4, App. C), all boxes per launch.
//
// Mesh convention: cell c of a box has its centre at (c + 1/2) dg in the
// box-local frame; a particle at x_loc has mesh coordinate u = x_loc/dg - 1/2.
// The padded potential holds the 2 ghost layers of FDA order 2 (indices -2..Ng+1
// stored at 0..Ng+3).
//
//  deposit       B^sCOLA (Sec. 3.4.1) and the boundary source delta' = delta -
//                Lap Phi_BCs (Eq. 62), by brick binning: k_deposit.cu.
//  pad           ghost layers of the potential <- D1(a_K) * shell (LEP, Eq. 23).
//  poisson       the zero-boundary solve of App. C on delta': dense DST-I along z,
//                along y, then along x with the division
//                by lambda_l + lambda_m + lambda_n (Eq. 71) and the inverse x
//                transform, then inverse y, then inverse z with the 8/(Ng+1)^3
//                scale (Eqs. 66-67), written into the padded potential.
//                Each pass is a pencil matrix product Y = S X with the sine
//                matrix S_li = sin(pi (l+1)(i+1)/(Ng+1)) held in shared memory.
//  interp        FDA-2 central gradient at the 8 CIC corners, CIC-weighted
//                (Sec. 3.4.2); u is clamped to [-1, Ng] with i0 <= Ng - 1.
//  kick_drift    the sCOLA kick (Eqs. 48, 54) and COLA drift (Eq. 53) fused
//                with the interpolation.
#include <algorithm>

#include "device_util.cuh"

namespace scola {

namespace {

// ------------------------------------------------------------------ pad
__global__ void __launch_bounds__(kChunk)
k_pad(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks,
      const float *__restrict__ shell, float *__restrict__ phi, float D1) {
    const Chunk ch = chunks[blockIdx.x];
    const BoxDesc &B = boxes[ch.box];
    const long long idx = (long long)ch.start + threadIdx.x;
    if (idx >= shell_count(B.Ng, B.gpad)) return;
    int pi, pj, pk;
    shell_coord(idx, B.Ng, B.gpad, pi, pj, pk);
    const long long S = B.Ng + 2 * B.gpad;
    phi[B.pp_off + ((long long)pi * S + pj) * S + pk] = D1 * shell[B.sh_off + idx];
}

// ------------------------------------------------------------------ DST passes
enum Pass { kYFwd = 1, kXSolve = 2, kYInv = 3, kZInv = 4, kZFwdF = 5 };

// acc[r][j] = sum_i ST[i][tl + 32 r] X[i][c0 + j]   (Y = S X on a column tile)
template <int R>
__device__ __forceinline__ void tile_product(const float *__restrict__ ST, int LS,
                                             const float *__restrict__ X, int Ng, int tl, int c0,
                                             float (&acc)[R][4]) {
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[r][j] = 0.0f;
#pragma unroll 4
    for (int i = 0; i < Ng; ++i) {
        const float4 xv = *reinterpret_cast<const float4 *>(X + i * kXS + c0);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float sv = ST[i * LS + tl + 32 * r];
            acc[r][0] = fmaf(sv, xv.x, acc[r][0]);
            acc[r][1] = fmaf(sv, xv.y, acc[r][1]);
            acc[r][2] = fmaf(sv, xv.z, acc[r][2]);
            acc[r][3] = fmaf(sv, xv.w, acc[r][3]);
        }
    }
}

template <int R, int PASS>
__global__ void __launch_bounds__(256)
k_dst(const BoxDesc *__restrict__ boxes, const DstTable *__restrict__ tables,
      const float *__restrict__ tab, const Chunk *__restrict__ items, int nitems,
      const void *__restrict__ in_v, float *__restrict__ out, const float *__restrict__ phi_pad,
      int ngmax) {
    // shared layout, sized for the largest Ng of the launch:
    //   ST[ngmax][32 R] | X[ngmax][kXS] | lambda[ngmax]
    extern __shared__ __align__(16) float smem[];
    const int LS = 32 * R;
    const int tid = threadIdx.x;
    const int tl = tid >> 3, c0 = (tid & 7) * 4;
    int cur_tbl = -1, Ng = 0;
    float *ST = smem;
    float *X = smem + (long long)ngmax * LS;
    float *lam = X + ngmax * kXS;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const Chunk item = items[it];
        const BoxDesc &B = boxes[item.box];
        if (B.tbl != cur_tbl) {
            __syncthreads();
            const DstTable T = tables[B.tbl];
            Ng = T.Ng;
            for (int q = tid; q < Ng * LS; q += blockDim.x) ST[q] = tab[T.st_off + q];
            for (int q = tid; q < Ng; q += blockDim.x) lam[q] = tab[T.lam_off + q];
            cur_tbl = B.tbl;
            __syncthreads();
        }
        const long long Ng2 = (long long)Ng * Ng;
        // box fields in registers: the stores below could otherwise force reloads
        const long long m_off = B.m_off, pp_off = B.pp_off;
        // ---- load the column tile X[t][c]
        int ncols;
        long long zp0 = 0;     // first pencil (z passes)
        int plane = 0, k0 = 0; // (plane, column offset) for y/x passes
        if (PASS == kZFwdF || PASS == kZInv) {
            zp0 = (long long)item.start * kTC;
            ncols = (int)min((long long)kTC, Ng2 - zp0);
            for (int q = tid; q < Ng * kTC; q += blockDim.x) {
                const int t = q % Ng, c = q / Ng;
                float v = 0.0f;
                if (c < ncols) {
                    const float *in = reinterpret_cast<const float *>(in_v);
                    v = in[m_off + (zp0 + c) * Ng + t];
                }
                X[t * kXS + c] = v;
            }
        } else {
            const int nct = (Ng + kTC - 1) / kTC;
            plane = item.start / nct;
            k0 = (item.start % nct) * kTC;
            ncols = min(kTC, Ng - k0);
            const float *in = reinterpret_cast<const float *>(in_v);
            // y passes: element (t = j, k) of plane i; x pass: element (t = i, k) of plane j
            const long long base = m_off + (PASS == kXSolve ? (long long)plane * Ng : (long long)plane * Ng2) + k0;
            const long long tstride = (PASS == kXSolve) ? Ng2 : Ng;
            for (int q = tid; q < Ng * kTC; q += blockDim.x) {
                const int c = q % kTC, t = q / kTC;
                X[t * kXS + c] = (c < ncols) ? in[base + t * tstride + c] : 0.0f;
            }
        }
        __syncthreads();

        float acc[R][4];
        tile_product<R>(ST, LS, X, Ng, tl, c0, acc);

        if (PASS == kXSolve) {
            // divide by the sum of eigenvalues (Eq. 71), then inverse x transform
            __syncthreads();
            const float lm = lam[plane];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int l = tl + 32 * r;
                if (l < Ng) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int c = c0 + j;
                        const float ln = (c < ncols) ? lam[k0 + c] : -1.0f;
                        X[l * kXS + c] = acc[r][j] / (lam[l] + lm + ln);
                    }
                }
            }
            __syncthreads();
            tile_product<R>(ST, LS, X, Ng, tl, c0, acc);
        }

        // ---- store
        if (PASS == kYFwd || PASS == kYInv || PASS == kXSolve) {
            const long long base = m_off + (PASS == kXSolve ? (long long)plane * Ng : (long long)plane * Ng2) + k0;
            const long long tstride = (PASS == kXSolve) ? Ng2 : Ng;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int l = tl + 32 * r;
                if (l < Ng) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (c0 + j < ncols) out[base + l * tstride + c0 + j] = acc[r][j];
                }
            }
        } else {
            // z passes: transpose through shared memory so that pencils are written contiguously
            __syncthreads();
            const float scale = (PASS == kZInv) ? 8.0f / ((float)(Ng + 1) * (Ng + 1) * (Ng + 1)) : 1.0f;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int l = tl + 32 * r;
                if (l < Ng) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) X[l * kXS + c0 + j] = acc[r][j] * scale;
                }
            }
            __syncthreads();
            for (int q = tid; q < Ng * kTC; q += blockDim.x) {
                const int t = q % Ng, c = q / Ng;
                if (c < ncols) {
                    const long long p = zp0 + c;
                    if (PASS == kZFwdF) {
                        out[m_off + p * Ng + t] = X[t * kXS + c];
                    } else {
                        const int G = B.gpad;
                        const long long S = Ng + 2 * G;
                        const int i = (int)(p / Ng), j = (int)(p % Ng);
                        out[pp_off + ((long long)(i + G) * S + (j + G)) * S + G + t] = X[t * kXS + c];
                    }
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ interpolation
// grad (stored potential) at a particle: the central gradient of FDA order ORDER at the 8
// CIC corners, CIC-interpolated.  The mesh coordinate is clamped to [-N_ghost,
// Ng + N_ghost - 1] and the lower corner capped at Ng + N_ghost - 2 (the gradient exists on
// the grid padded by N_ghost, Sec. 3.4.2).
template <int ORDER>
__device__ __forceinline__ void interpolate_force(const BoxDesc &B, const float *__restrict__ phi,
                                                  const int b[3], const float s[3], float F[3]) {
    const int Ng = B.Ng, G = B.gpad, ng = Fda<ORDER>::ng;
    int i0[3];
    float w[3][2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float u = fmaf(s[a], B.inv_dg, fmaf((float)b[a], B.q2u, 0.5f * B.q2u - 0.5f));
        u = fminf(fmaxf(u, -(float)ng), (float)(Ng + ng - 1));
        int fl = (int)floorf(u);
        fl = min(fl, Ng + ng - 2);
        i0[a] = fl;
        const float f = u - (float)fl;
        w[a][0] = 1.0f - f;
        w[a][1] = f;
    }
    const long long S1 = Ng + 2 * G, S2 = S1 * S1;
    const float *P = phi + B.pp_off + ((long long)(i0[0] + G) * S1 + (i0[1] + G)) * S1 + (i0[2] + G);
    if (ORDER == 2) {
        float core[2][2][2], xm[2][2], xp[2][2], ym[2][2], yp[2][2], zm[2][2], zp[2][2];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                for (int c = 0; c < 2; ++c) core[a][bb][c] = __ldg(P + a * S2 + bb * S1 + c);
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                xm[p][q] = __ldg(P - S2 + p * S1 + q);
                xp[p][q] = __ldg(P + 2 * S2 + p * S1 + q);
                ym[p][q] = __ldg(P + p * S2 - S1 + q);
                yp[p][q] = __ldg(P + p * S2 + 2 * S1 + q);
                zm[p][q] = __ldg(P + p * S2 + q * S1 - 1);
                zp[p][q] = __ldg(P + p * S2 + q * S1 + 2);
            }
        float fx = 0.0f, fy = 0.0f, fz = 0.0f;
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                // x gradient at corners (0|1, p, q)
                fx += w[1][p] * w[2][q] *
                      (w[0][0] * (core[1][p][q] - xm[p][q]) + w[0][1] * (xp[p][q] - core[0][p][q]));
                // y gradient at corners (p, 0|1, q)
                fy += w[0][p] * w[2][q] *
                      (w[1][0] * (core[p][1][q] - ym[p][q]) + w[1][1] * (yp[p][q] - core[p][0][q]));
                // z gradient at corners (p, q, 0|1)
                fz += w[0][p] * w[1][q] *
                      (w[2][0] * (core[p][q][1] - zm[p][q]) + w[2][1] * (zp[p][q] - core[p][q][0]));
            }
        const float h = 0.5f * B.inv_dg;
        F[0] = fx * h;
        F[1] = fy * h;
        F[2] = fz * h;
        return;
    }
    // orders 4 and 6: sum_m g_m (Phi(c + m e_a) - Phi(c - m e_a)) at every corner c
    const long long st[3] = {S2, S1, 1};
    float acc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int dx = 0; dx < 2; ++dx)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dz = 0; dz < 2; ++dz) {
                const float wc = w[0][dx] * w[1][dy] * w[2][dz];
                const float *C = P + dx * S2 + dy * S1 + dz;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    float g = 0.0f;
#pragma unroll
                    for (int m = 1; m <= Fda<ORDER>::ng; ++m)
                        g = fmaf(Fda<ORDER>::g(m), __ldg(C + m * st[a]) - __ldg(C - m * st[a]), g);
                    acc[a] = fmaf(wc, g, acc[a]);
                }
            }
#pragma unroll
    for (int a = 0; a < 3; ++a) F[a] = acc[a] * B.inv_dg;
}

template <int ORDER>
__global__ void __launch_bounds__(kChunk)
k_interp(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks,
         const float *__restrict__ s, long long stride, const float *__restrict__ phi, float D1,
         float *__restrict__ F) {
    const Chunk ch = chunks[blockIdx.x];
    const BoxDesc &B = boxes[ch.box];
    const int Nsc = B.Nsc;
    const int local = ch.start + threadIdx.x;
    if (local >= Nsc * Nsc * Nsc) return;
    const long long gi = B.p_off + local;
    int b[3];
    decode_local(local, Nsc, b[0], b[1], b[2]);
    float sv[3] = {s[gi], s[stride + gi], s[2 * stride + gi]};
    float f[3];
    interpolate_force<ORDER>(B, phi, b, sv, f);
    F[gi] = D1 * f[0];
    F[stride + gi] = D1 * f[1];
    F[2 * stride + gi] = D1 * f[2];
}

template <int ORDER>
__global__ void __launch_bounds__(kChunk, 5)
k_kick_drift(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks,
             float *__restrict__ part, long long P, const float *__restrict__ phi, KickDrift kd,
             int *__restrict__ kcount, const float *__restrict__ coef, int k, int nk) {
    const Chunk ch = chunks[blockIdx.x];
    const BoxDesc &B = boxes[ch.box];
    if (const float *c = box_coef(coef, ch.box, k, nk)) {     // this box's own time factors
        kd.kF = c[0];
        kd.k1 = c[1];
        kd.k2 = c[2];
        kd.alpha = c[3];
        kd.d1 = c[4];
        kd.d2 = c[5];
    }
    const int Nsc = B.Nsc;
    const int local = ch.start + threadIdx.x;
    int key = -1;
    if (local < Nsc * Nsc * Nsc) {
        const long long gi = B.p_off + local;
        int b[3];
        decode_local(local, Nsc, b[0], b[1], b[2]);
        float s[3], p[3], p1[3], p2[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            s[a] = part[a * P + gi];
            p[a] = part[(3 + a) * P + gi];
            p1[a] = __ldg(part + (6 + a) * P + gi);
            p2[a] = __ldg(part + (9 + a) * P + gi);
        }
        float F[3];
        interpolate_force<ORDER>(B, phi, b, s, F);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            p[a] = fmaf(kd.kF, F[a], fmaf(kd.k1, p1[a], fmaf(kd.k2, p2[a], p[a])));
            part[(3 + a) * P + gi] = p[a];
            if (kd.drift) {
                s[a] = fmaf(kd.alpha, p[a], fmaf(kd.d1, p1[a], fmaf(kd.d2, p2[a], s[a])));
                part[a * P + gi] = s[a];
            }
        }
        if (kcount) key = brick_entry(B, s, b).key;
    }
    // the next deposit's key counts (sorted form): one atomic per distinct key per warp
    if (kcount) {
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
        if (key >= 0 && lane == leader) atomicAdd(kcount + B.key_off + key, __popc(peers));
    }
}

size_t dst_smem_bytes(int R, int ngmax) {
    return ((size_t)ngmax * 32 * R + (size_t)ngmax * kXS + ngmax) * sizeof(float);
}

template <int R, int PASS>
cudaError_t run_pass(Ctx &c, const Chunk *items, int nitems, const void *in, float *out) {
    const size_t smem = dst_smem_bytes(R, c.max_ng);
    int grid = std::min(nitems, c.num_sms * c.dst_ctas_per_sm);
    if (grid < 1) grid = 1;
    k_dst<R, PASS><<<grid, 256, smem, c.stream>>>(c.boxes, c.tables, c.table_arena, items, nitems, in,
                                                   out, c.phi, c.max_ng);
    ++c.launches;
    return cudaGetLastError();
}

template <int R>
cudaError_t set_attrs_R() {
    const int lim = 227 * 1024;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_dst<R, kZFwdF>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(k_dst<R, kYFwd>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(k_dst<R, kXSolve>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(k_dst<R, kYInv>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    return cudaFuncSetAttribute(k_dst<R, kZInv>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

template <int R>
int ctas_per_sm_R(int ngmax) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_dst<R, kYFwd>, 256, dst_smem_bytes(R, ngmax)) !=
        cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

template <int R>
cudaError_t poisson_R(Ctx &c, const float *in, float *w1, float *w2, float *out_pad) {
    cudaError_t e;
    if ((e = run_pass<R, kZFwdF>(c, c.zitems, c.n_zitems, in, w1)) != cudaSuccess) return e;
    if ((e = run_pass<R, kYFwd>(c, c.citems, c.n_citems, w1, w2)) != cudaSuccess) return e;
    if ((e = run_pass<R, kXSolve>(c, c.citems, c.n_citems, w2, w1)) != cudaSuccess) return e;
    if ((e = run_pass<R, kYInv>(c, c.citems, c.n_citems, w1, w2)) != cudaSuccess) return e;
    return run_pass<R, kZInv>(c, c.zitems, c.n_zitems, w2, out_pad);
}

}  // namespace

cudaError_t launch_pad(Ctx &c, float D1) {
    k_pad<<<c.n_shchunks, kChunk, 0, c.stream>>>(c.boxes, c.shchunks, c.shell, c.phi, D1);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t init_pm_kernels(Ctx &c) {
    cudaError_t e;
    switch (c.max_R) {
        case 1: e = set_attrs_R<1>(); c.dst_ctas_per_sm = ctas_per_sm_R<1>(c.max_ng); break;
        case 2: e = set_attrs_R<2>(); c.dst_ctas_per_sm = ctas_per_sm_R<2>(c.max_ng); break;
        case 3: e = set_attrs_R<3>(); c.dst_ctas_per_sm = ctas_per_sm_R<3>(c.max_ng); break;
        case 4: e = set_attrs_R<4>(); c.dst_ctas_per_sm = ctas_per_sm_R<4>(c.max_ng); break;
        case 5: e = set_attrs_R<5>(); c.dst_ctas_per_sm = ctas_per_sm_R<5>(c.max_ng); break;
        case 6: e = set_attrs_R<6>(); c.dst_ctas_per_sm = ctas_per_sm_R<6>(c.max_ng); break;
        case 7:
            if (dst_smem_bytes(7, c.max_ng) > 227 * 1024) return cudaErrorInvalidValue;
            e = set_attrs_R<7>(); c.dst_ctas_per_sm = ctas_per_sm_R<7>(c.max_ng); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    if (dst_smem_bytes(c.max_R, c.max_ng) > 227 * 1024) return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t launch_poisson_buffers(Ctx &c, const float *in, float *w1, float *w2, float *out_pad) {
    if (c.rx) return launch_poisson_rx_buffers(c, in, w1, w2, out_pad);
    if (c.use_tc) return launch_poisson_tc_buffers(c, in, w1, w2, out_pad);
    switch (c.max_R) {
        case 1: return poisson_R<1>(c, in, w1, w2, out_pad);
        case 2: return poisson_R<2>(c, in, w1, w2, out_pad);
        case 3: return poisson_R<3>(c, in, w1, w2, out_pad);
        case 4: return poisson_R<4>(c, in, w1, w2, out_pad);
        case 5: return poisson_R<5>(c, in, w1, w2, out_pad);
        case 6: return poisson_R<6>(c, in, w1, w2, out_pad);
        case 7: return poisson_R<7>(c, in, w1, w2, out_pad);
        default: return cudaErrorInvalidValue;
    }
}

// The solve of the source the deposit left in work2, into the padded potential.
cudaError_t launch_poisson(Ctx &c) { return launch_poisson_buffers(c, c.work2, c.work, c.work2, c.phi); }

cudaError_t launch_poisson_pass(Ctx &c, int pass) {
    // the passes of launch_poisson, one at a time (for per-kernel timing); the FP32
    // form has five passes, the tensor-core and radix forms six
    if (c.rx) return launch_poisson_rx_pass(c, pass);
    if (c.use_tc) return launch_poisson_tc_pass(c, pass);
    if (pass == 5) return cudaSuccess;
    switch (c.max_R * 8 + pass) {
#define SCOLA_PASS_CASES(R)                                                                     \
    case R * 8 + 0: return run_pass<R, kZFwdF>(c, c.zitems, c.n_zitems, c.work2, c.work);       \
    case R * 8 + 1: return run_pass<R, kYFwd>(c, c.citems, c.n_citems, c.work, c.work2);        \
    case R * 8 + 2: return run_pass<R, kXSolve>(c, c.citems, c.n_citems, c.work2, c.work);      \
    case R * 8 + 3: return run_pass<R, kYInv>(c, c.citems, c.n_citems, c.work, c.work2);        \
    case R * 8 + 4: return run_pass<R, kZInv>(c, c.zitems, c.n_zitems, c.work2, c.phi);
        SCOLA_PASS_CASES(1)
        SCOLA_PASS_CASES(2)
        SCOLA_PASS_CASES(3)
        SCOLA_PASS_CASES(4)
        SCOLA_PASS_CASES(5)
        SCOLA_PASS_CASES(6)
        SCOLA_PASS_CASES(7)
#undef SCOLA_PASS_CASES
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_interp(Ctx &c, const float *s, long long stride, float *F, float D1) {
    switch (c.prm.fda_order) {
        case 4: k_interp<4><<<c.n_pchunks, kChunk, 0, c.stream>>>(c.boxes, c.pchunks, s, stride, c.phi, D1, F); break;
        case 6: k_interp<6><<<c.n_pchunks, kChunk, 0, c.stream>>>(c.boxes, c.pchunks, s, stride, c.phi, D1, F); break;
        default: k_interp<2><<<c.n_pchunks, kChunk, 0, c.stream>>>(c.boxes, c.pchunks, s, stride, c.phi, D1, F);
    }
    ++c.launches;
    return cudaGetLastError();
}

namespace {
__global__ void k_scaled_copy(const float *__restrict__ in, float *__restrict__ out, long long n, float a) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a * in[i];
}
}  // namespace

cudaError_t launch_scaled_copy(Ctx &c, const float *in, float *out, long long n, float a) {
    const long long g = (n + 255) / 256;
    k_scaled_copy<<<(int)(g < 8192 ? (g > 0 ? g : 1) : 8192), 256, 0, c.stream>>>(in, out, n, a);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_kick_drift(Ctx &c, const KickDrift &kd, bool count_keys, int k) {
    int *kc = count_keys && kd.drift ? c.kcount : nullptr;
    const float *coef = k >= 0 ? c.coef : nullptr;
    switch (c.prm.fda_order) {
        case 4:
            k_kick_drift<4><<<c.n_pchunks, kChunk, 0, c.stream>>>(c.boxes, c.pchunks, c.part, c.P, c.phi, kd, kc,
                                                                   coef, k, c.coef_nk);
            break;
        case 6:
            k_kick_drift<6><<<c.n_pchunks, kChunk, 0, c.stream>>>(c.boxes, c.pchunks, c.part, c.P, c.phi, kd, kc,
                                                                   coef, k, c.coef_nk);
            break;
        default:
            k_kick_drift<2><<<c.n_pchunks, kChunk, 0, c.stream>>>(c.boxes, c.pchunks, c.part, c.P, c.phi, kd, kc,
                                                                   coef, k, c.coef_nk);
    }
    ++c.launches;
    return cudaGetLastError();
}

}  // namespace scola
