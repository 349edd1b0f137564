// Adjoint (vector-Jacobian products) of the sCOLA forward run: the gradient of a loss of
// the final positions and momenta (or of the final density) with respect to the white noise.
//
// Start of the reverse sweep, tile particles only (buffer particles leave no output):
//   k_adj_final_xp  x = (q + s) mod L and p = p_res + c1 Psi1 + c2 Psi2 (L+, Eq. 55) give
//                   lam_s = lam_x, lam_p = lam_p, lam_Psi1 = c1 lam_p, lam_Psi2 = c2 lam_p
//   k_adj_final     lam_s = the periodic CIC adjoint of a final-density cotangent, from the
//                   particle state (the density-loss entry point)
//   k_density_vjp   the same periodic CIC adjoint over the global arrays: lam_x from x
//
// Per box particle the backward state is 5 rows of 3 x P floats (adj arena):
//   lam_s (0..2), lam_p (3..5), lam_Psi1 (6..8), lam_Psi2 (9..11), lam_F (12..14).
// Reverse KDK (App. B, Eqs. 53-54), at every force evaluation k = n .. 0:
//   drift  s += alpha p + d1 Psi1 + d2 Psi2   -> lam_p += alpha lam_s, lam_Psi += d lam_s
//   kick   p += kF F + k1 Psi1 + k2 Psi2      -> lam_F = kF lam_p,   lam_Psi += k lam_p
//   force  F(s_k): recomputed mesh potential at the checkpointed s_k, then
//     k_adj_interp   lam_s += (d weights / ds) (G . lam_F)   (direct term, clamp aware)
//                    lam_G += weights * lam_F   (3 channels interleaved per padded cell)
//     k_adj_div      lam_Phi = -div lam_G (transpose of the central difference);
//                    interior part -> Dirichlet solve (self-adjoint), ghosts kept
//     k_adj_shell    lam_shell += D1(a_k) (lam_Phi_ghost - boundary-source transpose)
//     k_adj_deposit  lam_s += (d deposit weights / ds) lam_delta'
// then L-: lam_Psi1 -= D1(a_i) lam_s, lam_Psi2 += D2(a_i) lam_s, scattered to the
// full-box arrays, and the shells' adjoint scattered to phi1 (trilinear transpose).
// The 2LPT and colouring adjoints (Fourier, symmetric operators) are in capi.cu.
// Accumulations shared between particles use FP32 atomics (sum order varies).
// FDA order n = 2, 4, 6 (Sec. 3.1): padded grids of G = n ghost layers per side, gradients of
// n / 2 central-difference terms; each transpose follows the forward kernel of the same order.
#include "device_util.cuh"

namespace scola {

namespace {

__device__ __forceinline__ void corner_setup(const BoxDesc &B, const int b[3], const float s[3],
                                             float lo, float hi, int cap, int i0[3], float f[3],
                                             float free_[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float u_raw = fmaf(s[a], B.inv_dg, fmaf((float)b[a], B.q2u, 0.5f * B.q2u - 0.5f));
        const float u = fminf(fmaxf(u_raw, lo), hi);
        free_[a] = (u == u_raw) ? 1.0f : 0.0f;
        int fl = (int)floorf(u);
        fl = min(fl, cap);
        i0[a] = fl;
        f[a] = u - (float)fl;
    }
}

// Final tile particles: lam_s = d(periodic CIC density)/dx^T lam_delta (Sec. 4.1).
__global__ void __launch_bounds__(kChunk)
k_adj_final(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks,
            const float *__restrict__ part, long long P, int Np, int Ntile, float dq, float L,
            const float *__restrict__ lam_delta, float *__restrict__ adj) {
    const Chunk ch = chunks[blockIdx.x];
    const BoxDesc &B = boxes[ch.box];
    const int lt = ch.start + threadIdx.x;
    if (lt >= Ntile * Ntile * Ntile) return;
    int ti, tj, tk;
    decode_local(lt, Ntile, ti, tj, tk);
    const int Nsc = B.Nsc;
    const long long gi = B.p_off + ((long long)(ti + B.Nbuf) * Nsc + (tj + B.Nbuf)) * Nsc + (tk + B.Nbuf);
    const int g[3] = {B.tx * Ntile + ti, B.ty * Ntile + tj, B.tz * Ntile + tk};
    const float invL = 1.0f / L, inv_d = (float)Np / L;
    int i0[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float xv = ((float)g[a] + 0.5f) * dq + part[a * P + gi];
        xv -= L * floorf(xv * invL);
        if (xv >= L) xv -= L;
        if (xv < 0.0f) xv += L;
        const float u = xv * inv_d - 0.5f;
        const float fl = floorf(u);
        i0[a] = (int)fl;
        f[a] = u - fl;
    }
    const long long NN = (long long)Np * Np;
    float lam[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int dx = 0; dx < 2; ++dx)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dz = 0; dz < 2; ++dz) {
                const float wx = dx ? f[0] : 1.f - f[0], wy = dy ? f[1] : 1.f - f[1],
                            wz = dz ? f[2] : 1.f - f[2];
                const float v = lam_delta[wrap(i0[0] + dx, Np) * NN + (long long)wrap(i0[1] + dy, Np) * Np +
                                          wrap(i0[2] + dz, Np)];
                lam[0] += (dx ? 1.f : -1.f) * wy * wz * v;
                lam[1] += wx * (dy ? 1.f : -1.f) * wz * v;
                lam[2] += wx * wy * (dz ? 1.f : -1.f) * v;
            }
#pragma unroll
    for (int a = 0; a < 3; ++a) adj[a * P + gi] = lam[a] * inv_d;
}

// Final tile particles from the cotangents of the global outputs x and p (either may be
// null = zero): the transposes of B.2's copy and of L+ (Eq. 55).
__global__ void __launch_bounds__(kChunk)
k_adj_final_xp(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks, long long P, int Np,
               int Ntile, const float *__restrict__ lam_x, const float *__restrict__ lam_p, float c1, float c2,
               const float *__restrict__ coefL, float *__restrict__ adj) {
    const Chunk ch = chunks[blockIdx.x];
    const BoxDesc &B = boxes[ch.box];
    if (coefL) {                       // L+ at this tile's own final scale factor
        c1 = coefL[2 * ch.box];
        c2 = coefL[2 * ch.box + 1];
    }
    const int lt = ch.start + threadIdx.x;
    if (lt >= Ntile * Ntile * Ntile) return;
    int ti, tj, tk;
    decode_local(lt, Ntile, ti, tj, tk);
    const int Nsc = B.Nsc;
    const long long gi = B.p_off + ((long long)(ti + B.Nbuf) * Nsc + (tj + B.Nbuf)) * Nsc + (tk + B.Nbuf);
    const long long gid = ((long long)(B.tx * Ntile + ti) * Np + (B.ty * Ntile + tj)) * Np + (B.tz * Ntile + tk);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lp = lam_p ? lam_p[gid * 3 + a] : 0.0f;
        adj[a * P + gi] = lam_x ? lam_x[gid * 3 + a] : 0.0f;
        adj[(3 + a) * P + gi] = lp;
        adj[(6 + a) * P + gi] = c1 * lp;
        adj[(9 + a) * P + gi] = c2 * lp;
    }
}

// lam_x = d(periodic CIC density on the Np^3 grid)/dx^T lam_delta for every particle
// (Sec. 4.1), from the global positions; the same arithmetic as k_adj_final.
__global__ void k_density_vjp(const float *__restrict__ x, long long n, int Np, float inv_d,
                              const float *__restrict__ lam_delta, float *__restrict__ lam_x) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        int i0[3];
        float f[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float u = x[idx * 3 + a] * inv_d - 0.5f;
            const float fl = floorf(u);
            i0[a] = (int)fl;
            f[a] = u - fl;
        }
        const long long NN = (long long)Np * Np;
        float lam[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int dx = 0; dx < 2; ++dx)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dz = 0; dz < 2; ++dz) {
                    const float wx = dx ? f[0] : 1.f - f[0], wy = dy ? f[1] : 1.f - f[1],
                                wz = dz ? f[2] : 1.f - f[2];
                    const float v = lam_delta[wrap(i0[0] + dx, Np) * NN + (long long)wrap(i0[1] + dy, Np) * Np +
                                              wrap(i0[2] + dz, Np)];
                    lam[0] += (dx ? 1.f : -1.f) * wy * wz * v;
                    lam[1] += wx * (dy ? 1.f : -1.f) * wz * v;
                    lam[2] += wx * wy * (dz ? 1.f : -1.f) * v;
                }
#pragma unroll
        for (int a = 0; a < 3; ++a) lam_x[idx * 3 + a] = lam[a] * inv_d;
    }
}

__global__ void __launch_bounds__(kChunk)
k_adj_kick_drift(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks,
                 float *__restrict__ adj, long long P, KickDrift kd, const float *__restrict__ coef, int k, int nk) {
    const Chunk ch = chunks[blockIdx.x];
    const BoxDesc &B = boxes[ch.box];
    if (const float *cf = box_coef(coef, ch.box, k, nk)) {     // this box's own time factors
        kd.kF = cf[7];
        kd.k1 = cf[1];
        kd.k2 = cf[2];
        kd.alpha = cf[3];
        kd.d1 = cf[4];
        kd.d2 = cf[5];
    }
    const int local = ch.start + threadIdx.x;
    if (local >= B.Nsc * B.Nsc * B.Nsc) return;
    const long long gi = B.p_off + local;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float ls = adj[a * P + gi];
        float lp = adj[(3 + a) * P + gi];
        float l1 = adj[(6 + a) * P + gi];
        float l2 = adj[(9 + a) * P + gi];
        if (kd.drift) {
            lp = fmaf(kd.alpha, ls, lp);
            l1 = fmaf(kd.d1, ls, l1);
            l2 = fmaf(kd.d2, ls, l2);
        }
        l1 = fmaf(kd.k1, lp, l1);
        l2 = fmaf(kd.k2, lp, l2);
        adj[(3 + a) * P + gi] = lp;
        adj[(6 + a) * P + gi] = l1;
        adj[(9 + a) * P + gi] = l2;
        adj[(12 + a) * P + gi] = kd.kF * lp;
    }
}

template <int ORDER>
__global__ void __launch_bounds__(kChunk)
k_adj_interp(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks,
             const float *__restrict__ s, long long P, const float *__restrict__ phi, float D1,
             float *__restrict__ adj, float *__restrict__ lamG, long long MP, const float *__restrict__ coef,
             int k, int nk) {
    const Chunk ch = chunks[blockIdx.x];
    const BoxDesc &B = boxes[ch.box];
    if (const float *cf = box_coef(coef, ch.box, k, nk)) D1 = 1.0f / cf[6];
    const int Nsc = B.Nsc, Ng = B.Ng, G = B.gpad, ng = Fda<ORDER>::ng;
    const int local = ch.start + threadIdx.x;
    if (local >= Nsc * Nsc * Nsc) return;
    const long long gi = B.p_off + local;
    int b[3];
    decode_local(local, Nsc, b[0], b[1], b[2]);
    const float sv[3] = {s[gi], s[P + gi], s[2 * P + gi]};
    const float lF[3] = {adj[12 * P + gi], adj[13 * P + gi], adj[14 * P + gi]};
    int i0[3];
    float f[3], fr[3];
    // the forward clamp: mesh coordinate in [-ng, Ng + ng - 1], lower corner <= Ng + ng - 2
    corner_setup(B, b, sv, -(float)ng, (float)(Ng + ng - 1), Ng + ng - 2, i0, f, fr);
    const long long S1 = Ng + 2 * G, S2 = S1 * S1;
    const long long st[3] = {S2, S1, 1};
    const long long base = B.pp_off + ((long long)(i0[0] + G) * S1 + (i0[1] + G)) * S1 + (i0[2] + G);
    const float *Pp = phi + base;
    const float h = B.inv_dg * D1;            // the stored potential is Phi / D1
    float dir[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int dx = 0; dx < 2; ++dx)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dz = 0; dz < 2; ++dz) {
                const long long o = dx * S2 + dy * S1 + dz;
                float gl = 0.0f;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    float g = 0.0f;
#pragma unroll
                    for (int m = 1; m <= ng; ++m) g = fmaf(Fda<ORDER>::g(m), Pp[o + m * st[a]] - Pp[o - m * st[a]], g);
                    gl = fmaf(g * h, lF[a], gl);
                }
                const float wx = dx ? f[0] : 1.f - f[0], wy = dy ? f[1] : 1.f - f[1],
                            wz = dz ? f[2] : 1.f - f[2];
                dir[0] += (dx ? 1.f : -1.f) * wy * wz * gl;
                dir[1] += wx * (dy ? 1.f : -1.f) * wz * gl;
                dir[2] += wx * wy * (dz ? 1.f : -1.f) * gl;
                const float w = wx * wy * wz;
                // lam_G interleaved per padded cell (x, y, z, unused): one 16-byte vector atomic
                atomicAdd(reinterpret_cast<float4 *>(lamG) + base + o, make_float4(w * lF[0], w * lF[1], w * lF[2], 0.f));
            }
#pragma unroll
    for (int a = 0; a < 3; ++a) adj[a * P + gi] += dir[a] * fr[a] * B.inv_dg;
}

// lam_Phi(c) = sum_a sum_m g_m (lam_G_a(c - m e_a) - lam_G_a(c + m e_a)) / dg over the padded grid
// (the transpose of the order-n central gradient); lam_G interleaved, one float4 per cell.
template <int ORDER>
__global__ void __launch_bounds__(kChunk)
k_adj_div(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks,
          const float *__restrict__ lamG, long long MP, float *__restrict__ lam_phi_pad,
          float *__restrict__ interior_out) {
    const Chunk ch = chunks[blockIdx.x];
    const BoxDesc &B = boxes[ch.box];
    const int Ng = B.Ng, G = B.gpad, S = Ng + 2 * G;
    const long long n = (long long)S * S * S;
    const long long idx = (long long)ch.start + threadIdx.x;
    if (idx >= n) return;
    int p[3];
    decode_local((int)idx, S, p[0], p[1], p[2]);
    const long long strides[3] = {(long long)S * S, S, 1};
    const long long here = B.pp_off + idx;
    float v = 0.0f;
    const float *G4 = lamG;          // 4 floats per padded cell
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int m = 1; m <= Fda<ORDER>::ng; ++m) {
            float d = 0.0f;
            if (p[a] - m >= 0) d += G4[4 * (here - m * strides[a]) + a];
            if (p[a] + m < S) d -= G4[4 * (here + m * strides[a]) + a];
            v = fmaf(Fda<ORDER>::g(m), d, v);
        }
    }
    v *= B.inv_dg;
    const bool inside = p[0] >= G && p[0] < Ng + G && p[1] >= G && p[1] < Ng + G && p[2] >= G && p[2] < Ng + G;
    if (inside)
        interior_out[B.m_off + ((long long)(p[0] - G) * Ng + (p[1] - G)) * Ng + (p[2] - G)] = v;
    else
        lam_phi_pad[here] = v;
}

// lam_shell += D1 (lam_Phi_ghost - transpose of the boundary source of Eq. 62).  A ghost
// cell m' layers beyond a face, whose other two coordinates are interior, enters the order-n
// Laplacian of the interior cells m - m' from the face (m = m' .. n / 2) with weight s_m.
template <int ORDER>
__global__ void __launch_bounds__(kChunk)
k_adj_shell(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks,
            const float *__restrict__ lam_phi_pad, const float *__restrict__ lam_src_pad, float D1,
            float *__restrict__ lam_shell, const float *__restrict__ coef, int k, int nk) {
    const Chunk ch = chunks[blockIdx.x];
    const BoxDesc &B = boxes[ch.box];
    if (const float *cf = box_coef(coef, ch.box, k, nk)) D1 = 1.0f / cf[6];
    const int Ng = B.Ng, G = B.gpad;
    const long long idx = (long long)ch.start + threadIdx.x;
    if (idx >= shell_count(Ng, G)) return;
    int p[3];
    shell_coord(idx, Ng, G, p[0], p[1], p[2]);
    const long long S = Ng + 2 * G;
    const long long strides[3] = {S * S, S, 1};
    const long long here = B.pp_off + ((long long)p[0] * S + p[1]) * S + p[2];
    float v = lam_phi_pad[here];
    const float c2 = B.inv_dg * B.inv_dg;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int o1 = (a + 1) % 3, o2 = (a + 2) % 3;
        const bool others = p[o1] >= G && p[o1] < Ng + G && p[o2] >= G && p[o2] < Ng + G;
        if (!others) continue;
        const int below = G - p[a], above = p[a] - (Ng + G - 1);      // m' on either side
#pragma unroll
        for (int m = 1; m <= Fda<ORDER>::ng; ++m) {
            if (below >= 1 && m >= below) v -= Fda<ORDER>::s(m) * lam_src_pad[here + m * strides[a]] * c2;
            if (above >= 1 && m >= above) v -= Fda<ORDER>::s(m) * lam_src_pad[here - m * strides[a]] * c2;
        }
    }
    lam_shell[B.sh_off + idx] += D1 * v;
}

__global__ void __launch_bounds__(kChunk)
k_adj_deposit(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks,
              const float *__restrict__ s, long long P, const float *__restrict__ lam_src_pad,
              float *__restrict__ adj) {
    const Chunk ch = chunks[blockIdx.x];
    const BoxDesc &B = boxes[ch.box];
    const int Nsc = B.Nsc, Ng = B.Ng;
    const int local = ch.start + threadIdx.x;
    if (local >= Nsc * Nsc * Nsc) return;
    const long long gi = B.p_off + local;
    int b[3];
    decode_local(local, Nsc, b[0], b[1], b[2]);
    const float sv[3] = {s[gi], s[P + gi], s[2 * P + gi]};
    int i0[3];
    float f[3], fr[3];
    corner_setup(B, b, sv, -2.0f, (float)Ng + 1.0f, Ng + 1, i0, f, fr);
    const int G = B.gpad;
    const long long S = Ng + 2 * G;
    float lam[3] = {0.f, 0.f, 0.f};
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
                if ((unsigned)cz >= (unsigned)Ng) continue;
                const float v = lam_src_pad[B.pp_off + ((long long)(cx + G) * S + (cy + G)) * S + (cz + G)];
                const float wx = dx ? f[0] : 1.f - f[0], wy = dy ? f[1] : 1.f - f[1],
                            wz = dz ? f[2] : 1.f - f[2];
                lam[0] += (dx ? 1.f : -1.f) * wy * wz * v;
                lam[1] += wx * (dy ? 1.f : -1.f) * wz * v;
                lam[2] += wx * wy * (dz ? 1.f : -1.f) * v;
            }
        }
    }
    const float sc = B.nbar_inv * B.inv_dg;
#pragma unroll
    for (int a = 0; a < 3; ++a) adj[a * P + gi] += lam[a] * sc * fr[a];
}

// L- adjoint and scatter of lam_Psi1, lam_Psi2 to the full-box arrays (3 x N^3 each).
__global__ void __launch_bounds__(kChunk)
k_adj_init_scatter(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks,
                   const float *__restrict__ adj, long long P, int Np, int Ntile, long long N3,
                   float D1i, float D2i, float *__restrict__ lamPsi1, float *__restrict__ lamPsi2) {
    const Chunk ch = chunks[blockIdx.x];
    const BoxDesc &B = boxes[ch.box];
    const int Nsc = B.Nsc;
    const int local = ch.start + threadIdx.x;
    if (local >= Nsc * Nsc * Nsc) return;
    const long long gi = B.p_off + local;
    int bi, bj, bk;
    decode_local(local, Nsc, bi, bj, bk);
    const int gx = wrap(B.tx * Ntile - B.Nbuf + bi, Np);
    const int gy = wrap(B.ty * Ntile - B.Nbuf + bj, Np);
    const int gz = wrap(B.tz * Ntile - B.Nbuf + bk, Np);
    const long long gid = ((long long)gx * Np + gy) * Np + gz;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float ls = adj[a * P + gi];
        atomicAdd(lamPsi1 + a * N3 + gid, adj[(6 + a) * P + gi] - D1i * ls);
        atomicAdd(lamPsi2 + a * N3 + gid, adj[(9 + a) * P + gi] + D2i * ls);
    }
}

// Trilinear transpose of C.3: lam_phi1 += sum over shell cells of weights * lam_shell.
__global__ void __launch_bounds__(kChunk)
k_adj_shell_to_phi1(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks,
                    const float *__restrict__ lam_shell, int N, int Ntile,
                    float *__restrict__ lam_phi1) {
    const Chunk ch = chunks[blockIdx.x];
    const BoxDesc &B = boxes[ch.box];
    const long long idx = (long long)ch.start + threadIdx.x;
    if (idx >= shell_count(B.Ng, B.gpad)) return;
    const float lv = lam_shell[B.sh_off + idx];
    if (lv == 0.0f) return;
    int pc[3];
    shell_coord(idx, B.Ng, B.gpad, pc[0], pc[1], pc[2]);
    int i0[3];
    float f[3];
    shell_stencil(B, pc, Ntile, i0, f);
    const long long NN = (long long)N * N;
#pragma unroll
    for (int dx = 0; dx < 2; ++dx)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dz = 0; dz < 2; ++dz) {
                const float w = (dx ? f[0] : 1.0f - f[0]) * (dy ? f[1] : 1.0f - f[1]) * (dz ? f[2] : 1.0f - f[2]);
                atomicAdd(lam_phi1 + wrap(i0[0] + dx, N) * NN + (long long)wrap(i0[1] + dy, N) * N +
                              wrap(i0[2] + dz, N),
                          w * lv);
            }
}

// out = -sum_a D_a(g_a) (+ out when accumulate): the transpose of the periodic order-n central
// gradient D_a f(c) = (1/d) sum_m g_m (f(c + m e_a) - f(c - m e_a)).
template <int ORDER>
__global__ void k_neg_div(const float *__restrict__ g, int N, float inv_d, int accumulate, float *__restrict__ out) {
    const long long N3 = (long long)N * N * N, NN = (long long)N * N;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N3;
         idx += (long long)gridDim.x * blockDim.x) {
        const int c[3] = {(int)(idx / NN), (int)((idx / N) % N), (int)(idx % N)};
        const long long st[3] = {NN, N, 1};
        float v = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float *ga = g + a * N3;
            const long long rest = idx - c[a] * st[a];
#pragma unroll
            for (int m = 1; m <= Fda<ORDER>::ng; ++m)
                v = fmaf(Fda<ORDER>::g(m), ga[rest + wrap(c[a] + m, N) * st[a]] - ga[rest + wrap(c[a] - m, N) * st[a]], v);
        }
        out[idx] = (accumulate ? out[idx] : 0.0f) - v * inv_d;
    }
}

// lam_ij products of the second-order source (transpose of Eq. 6's bilinear form).
__global__ void k_adj_source(const float *__restrict__ lamS, const float *__restrict__ d2, long long n,
                             float *__restrict__ lam_d2) {
    // d2: xx, yy, zz, xy, xz, yz (6 x n); lam_d2 same layout
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float ls = lamS[i];
        const float xx = d2[i], yy = d2[n + i], zz = d2[2 * n + i];
        lam_d2[i] = ls * (yy + zz);
        lam_d2[n + i] = ls * (xx + zz);
        lam_d2[2 * n + i] = ls * (xx + yy);
        lam_d2[3 * n + i] = -2.0f * ls * d2[3 * n + i];
        lam_d2[4 * n + i] = -2.0f * ls * d2[4 * n + i];
        lam_d2[5 * n + i] = -2.0f * ls * d2[5 * n + i];
    }
}

// acc_hat += (-D_i D_j) in_hat  (spectral second derivative, symmetric)
__global__ void k_spec_d2_accumulate(const cufftComplex *__restrict__ in, cufftComplex *__restrict__ acc,
                                     int N, const float *__restrict__ s_full, int ai, int aj) {
    const int Nz = N / 2 + 1;
    const long long n = (long long)N * N * Nz;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        int c[3];
        c[2] = (int)(idx % Nz);
        const long long t = idx / Nz;
        c[1] = (int)(t % N);
        c[0] = (int)(t / N);
        const float m = -s_full[c[ai]] * s_full[c[aj]];
        cufftComplex a = acc[idx];
        const cufftComplex v = in[idx];
        a.x = fmaf(m, v.x, a.x);
        a.y = fmaf(m, v.y, a.y);
        acc[idx] = a;
    }
}

int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    return (int)(g < 8192 ? (g > 0 ? g : 1) : 8192);
}

}  // namespace

cudaError_t launch_adj_final(Ctx &c, const float *lam_delta, float *adj) {
    const int Ntile = c.Np / c.Ntiles;
    k_adj_final<<<c.n_tchunks, kChunk, 0, c.stream>>>(c.boxes, c.tchunks, c.part, c.P, c.Np, Ntile,
                                                       (float)c.dq, (float)c.L, lam_delta, adj);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_adj_final_xp(Ctx &c, const float *lam_x, const float *lam_p, float *adj) {
    const int Ntile = c.Np / c.Ntiles;
    const double af = c.prm.a_f;
    const double pref = af * af * c.tt.Hconf_f;
    k_adj_final_xp<<<c.n_tchunks, kChunk, 0, c.stream>>>(c.boxes, c.tchunks, c.P, c.Np, Ntile, lam_x, lam_p,
                                                          (float)(-pref * c.tt.dD1da_f),
                                                          (float)(pref * c.tt.dD2da_f), c.coefL, adj);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_density_vjp(Ctx &c, const float *x, const float *lam_delta, float *lam_x) {
    k_density_vjp<<<grid_for(c.N3, 256), 256, 0, c.stream>>>(x, c.N3, c.Np, (float)((double)c.Np / c.L), lam_delta,
                                                             lam_x);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_adj_kick_drift(Ctx &c, float *adj, const KickDrift &kd, int k) {
    k_adj_kick_drift<<<c.n_pchunks, kChunk, 0, c.stream>>>(c.boxes, c.pchunks, adj, c.P, kd,
                                                            k >= 0 ? c.coef : nullptr, k, c.coef_nk);
    ++c.launches;
    return cudaGetLastError();
}

// the kernel template of the context's FDA order
#define SCOLA_BY_ORDER(KERNEL, GRID, ...)                                                    \
    switch (c.prm.fda_order) {                                                               \
        case 4: KERNEL<4><<<GRID, kChunk, 0, c.stream>>>(__VA_ARGS__); break;                \
        case 6: KERNEL<6><<<GRID, kChunk, 0, c.stream>>>(__VA_ARGS__); break;                \
        default: KERNEL<2><<<GRID, kChunk, 0, c.stream>>>(__VA_ARGS__);                      \
    }

cudaError_t launch_adj_interp(Ctx &c, const float *s, float *adj, float *lamG, float D1, int k) {
    SCOLA_BY_ORDER(k_adj_interp, c.n_pchunks, c.boxes, c.pchunks, s, c.P, c.phi, D1, adj, lamG, c.MP,
                   k >= 0 ? c.coef : nullptr, k, c.coef_nk)
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_adj_div(Ctx &c, const float *lamG, float *lam_phi_pad, float *interior_out) {
    SCOLA_BY_ORDER(k_adj_div, c.n_ppchunks, c.boxes, c.ppchunks, lamG, c.MP, lam_phi_pad, interior_out)
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_adj_shell(Ctx &c, const float *lam_phi_pad, const float *lam_src_pad, float D1,
                             float *lam_shell, int k) {
    SCOLA_BY_ORDER(k_adj_shell, c.n_shchunks, c.boxes, c.shchunks, lam_phi_pad, lam_src_pad, D1, lam_shell,
                   k >= 0 ? c.coef : nullptr, k, c.coef_nk)
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_adj_deposit(Ctx &c, const float *s, const float *lam_src_pad, float *adj) {
    k_adj_deposit<<<c.n_pchunks, kChunk, 0, c.stream>>>(c.boxes, c.pchunks, s, c.P, lam_src_pad, adj);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_adj_init_scatter(Ctx &c, const float *adj, float *lamPsi1, float *lamPsi2) {
    const int Ntile = c.Np / c.Ntiles;
    k_adj_init_scatter<<<c.n_pchunks, kChunk, 0, c.stream>>>(c.boxes, c.pchunks, adj, c.P, c.Np, Ntile, c.N3,
                                                              (float)c.tt.D1_i, (float)c.tt.D2_i, lamPsi1,
                                                              lamPsi2);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_adj_shell_to_phi1(Ctx &c, const float *lam_shell, float *lam_phi1) {
    k_adj_shell_to_phi1<<<c.n_shchunks, kChunk, 0, c.stream>>>(c.boxes, c.shchunks, lam_shell, c.Np,
                                                                c.Np / c.Ntiles, lam_phi1);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_neg_div(Ctx &c, const float *g, int accumulate, float *out) {
    const float inv_d = (float)(c.Np / c.L);
    const int grid = grid_for(c.N3, 256);
    switch (c.prm.fda_order) {
        case 4: k_neg_div<4><<<grid, 256, 0, c.stream>>>(g, c.Np, inv_d, accumulate, out); break;
        case 6: k_neg_div<6><<<grid, 256, 0, c.stream>>>(g, c.Np, inv_d, accumulate, out); break;
        default: k_neg_div<2><<<grid, 256, 0, c.stream>>>(g, c.Np, inv_d, accumulate, out);
    }
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_adj_source(Ctx &c, const float *lamS, const float *d2, float *lam_d2) {
    k_adj_source<<<grid_for(c.N3, 256), 256, 0, c.stream>>>(lamS, d2, c.N3, lam_d2);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_spec_d2_accumulate(Ctx &c, const cufftComplex *in, cufftComplex *acc, int i, int j) {
    const int N = c.Np;
    const long long n = (long long)N * N * (N / 2 + 1);
    // the gradient symbol of the context's FDA order (as the forward second derivatives)
    k_spec_d2_accumulate<<<grid_for(n, 256), 256, 0, c.stream>>>(
        in, acc, N, c.table_arena + (c.prm.fda_order != 2 ? c.grad1_off : c.sin_full_off), i, j);
    ++c.launches;
    return cudaGetLastError();
}

}  // namespace scola
