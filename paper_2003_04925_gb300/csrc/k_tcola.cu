// Periodic full-box tCOLA (Sec. 2.2, App. A-B) and the approximation-study inputs of the
// boxes (Sec. 4.3).
//
// tCOLA is the monolithic simulation that sCOLA approximates: all Np^3 particles on one
// periodic PM grid of Ngf = mesh_ratio * Np cells per side, cell c centred at (c + 1/2) dg,
// dg = L / Ngf (the cells of every box mesh are cells of this grid), and the KDK factors of
// the boxes.  Particle state: s and p_res as SoA rows of N3 floats, global-id order.
//   init        s = -D1(a_i) Psi1 + D2(a_i) Psi2, p_res = 0 (Eqs. 39, 55)
//   deposit     periodic CIC, 2^-32 fixed-point 64-bit atomics (the sums do not depend on
//               the order of the additions: deterministic)
//   density     delta = (Ngf / Np)^3 n - 1; the counts are cleared as they are read
//   poisson     Phi_k = delta_k / (Lambda(k) Ngf^3), Lambda the FDA-2 Laplacian symbol
//               sum_a (2 / dg^2)(cos(k_a dg) - 1), k = 0 removed (k_tcola_fft.cu: five passes
//               of shared-memory FFTs)
//   kick_drift  FDA-2 central gradient at the 8 CIC corners (periodic wrap), CIC-weighted,
//               then the kick (Eqs. 48, 54) and the drift (Eq. 53)
//   final       x = (q + s) mod L, p = p_res + L+ at a_f (Eq. 55)
// Study inputs (Sec. 4.3), per force evaluation K, for every box of the bound batch:
//   true source     delta_int = the recorded delta_K restricted to the box interior: the
//                   Poisson source delta_K / D1(a_K) minus the boundary term of the ghost
//                   layers (in place of the deposit, Eq. 62)
//   true potential  Phi_BCs = the recorded Phi_K restricted to the ghost layers, stored
//                   as Phi_K / D1(a_K) like the rest of the padded potential (in place of
//                   the LEP shell, Eq. 23)
// A box cell c (interior index, or padded index minus the ghost width) is full-grid cell
// (t Ntile - Nbuf) mesh_ratio + c, wrapped: the restriction is a copy by index.
#include "device_util.cuh"

namespace scola {

namespace {

__device__ __forceinline__ void gid_coords(long long gid, int Np, int g[3]) {
    g[2] = (int)(gid % Np);
    const long long t = gid / Np;
    g[1] = (int)(t % Np);
    g[0] = (int)(t / Np);
}

// Mesh coordinate of a particle: u = x / dg - 1/2 with x = (g + 1/2) dq + s.
__device__ __forceinline__ float mesh_u(int g, float s, float q2u, float inv_dg) {
    return fmaf(s, inv_dg, fmaf((float)g, q2u, 0.5f * q2u - 0.5f));
}

__global__ void k_tc_init(float *__restrict__ part, const float *__restrict__ psi1, const float *__restrict__ psi2,
                          long long N3, float D1i, float D2i) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N3;
         i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float q1 = psi1[a * N3 + i], q2 = psi2[a * N3 + i];
            part[a * N3 + i] = -D1i * q1 + D2i * q2;
            part[(3 + a) * N3 + i] = 0.0f;
        }
    }
}

__global__ void k_tc_deposit(const float *__restrict__ part, long long N3, int Np, int Ngf, float q2u,
                             float inv_dg, unsigned long long *__restrict__ acc) {
    const long long NN = (long long)Ngf * Ngf;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N3;
         i += (long long)gridDim.x * blockDim.x) {
        int g[3];
        gid_coords(i, Np, g);
        int i0[3];
        float f[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float u = mesh_u(g[a], part[a * N3 + i], q2u, inv_dg);
            const float fl = floorf(u);
            i0[a] = (int)fl;
            f[a] = u - fl;
        }
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            const long long cx = wrap(i0[0] + dx, Ngf);
            const float wx = dx ? f[0] : 1.0f - f[0];
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                const long long cy = wrap(i0[1] + dy, Ngf);
                const float wxy = wx * (dy ? f[1] : 1.0f - f[1]);
#pragma unroll
                for (int dz = 0; dz < 2; ++dz) {
                    const long long cz = wrap(i0[2] + dz, Ngf);
                    const float w = wxy * (dz ? f[2] : 1.0f - f[2]);
                    atomicAdd(acc + cx * NN + cy * Ngf + cz, weight_to_fixed(w));
                }
            }
        }
    }
}

__global__ void k_tc_density(unsigned long long *__restrict__ acc, long long n, float sc, float *__restrict__ delta) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        delta[i] = fixed_to_float(acc[i]) * sc - 1.0f;
        acc[i] = 0ull;
    }
}

__global__ void __launch_bounds__(256)
k_tc_kick_drift(float *__restrict__ part, const float *__restrict__ psi1, const float *__restrict__ psi2,
                long long N3, int Np, int Ngf, float q2u, float inv_dg, const float *__restrict__ phi, KickDrift kd) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N3) return;
    int g[3];
    gid_coords(i, Np, g);
    float s[3], p[3], p1[3], p2[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        s[a] = part[a * N3 + i];
        p[a] = part[(3 + a) * N3 + i];
        p1[a] = __ldg(psi1 + a * N3 + i);
        p2[a] = __ldg(psi2 + a * N3 + i);
    }
    // wrapped indices i0 - 1 .. i0 + 2 per axis and the CIC weights
    long long ix[4], iy[4], iz[4];
    float w[3][2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float u = mesh_u(g[a], s[a], q2u, inv_dg);
        const float fl = floorf(u);
        const int i0 = (int)fl;
        const float f = u - fl;
        w[a][0] = 1.0f - f;
        w[a][1] = f;
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const long long v = wrap(i0 - 1 + o, Ngf);
            if (a == 0) ix[o] = v * Ngf * Ngf;
            if (a == 1) iy[o] = v * Ngf;
            if (a == 2) iz[o] = v;
        }
    }
    auto at = [&](int x, int y, int z) { return __ldg(phi + ix[x] + iy[y] + iz[z]); };
    float fx = 0.0f, fy = 0.0f, fz = 0.0f;
#pragma unroll
    for (int p0 = 0; p0 < 2; ++p0)
#pragma unroll
        for (int q0 = 0; q0 < 2; ++q0) {
            // x gradient at corners (0|1, p0, q0); y at (p0, 0|1, q0); z at (p0, q0, 0|1)
            fx += w[1][p0] * w[2][q0] *
                  (w[0][0] * (at(2, p0 + 1, q0 + 1) - at(0, p0 + 1, q0 + 1)) +
                   w[0][1] * (at(3, p0 + 1, q0 + 1) - at(1, p0 + 1, q0 + 1)));
            fy += w[0][p0] * w[2][q0] *
                  (w[1][0] * (at(p0 + 1, 2, q0 + 1) - at(p0 + 1, 0, q0 + 1)) +
                   w[1][1] * (at(p0 + 1, 3, q0 + 1) - at(p0 + 1, 1, q0 + 1)));
            fz += w[0][p0] * w[1][q0] *
                  (w[2][0] * (at(p0 + 1, q0 + 1, 2) - at(p0 + 1, q0 + 1, 0)) +
                   w[2][1] * (at(p0 + 1, q0 + 1, 3) - at(p0 + 1, q0 + 1, 1)));
        }
    const float h = 0.5f * inv_dg;
    const float F[3] = {fx * h, fy * h, fz * h};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        p[a] = fmaf(kd.kF, F[a], fmaf(kd.k1, p1[a], fmaf(kd.k2, p2[a], p[a])));
        part[(3 + a) * N3 + i] = p[a];
        if (kd.drift) part[a * N3 + i] = fmaf(kd.alpha, p[a], fmaf(kd.d1, p1[a], fmaf(kd.d2, p2[a], s[a])));
    }
}

__global__ void k_tc_final(const float *__restrict__ part, const float *__restrict__ psi1,
                           const float *__restrict__ psi2, long long N3, int Np, float dq, float L, float c1, float c2,
                           float *__restrict__ x, float *__restrict__ p) {
    const float invL = 1.0f / L;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N3;
         i += (long long)gridDim.x * blockDim.x) {
        int g[3];
        gid_coords(i, Np, g);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float xv = ((float)g[a] + 0.5f) * dq + part[a * N3 + i];
            xv -= L * floorf(xv * invL);
            if (xv >= L) xv -= L;
            if (xv < 0.0f) xv += L;
            x[i * 3 + a] = xv;
            p[i * 3 + a] = part[(3 + a) * N3 + i] + c1 * psi1[a * N3 + i] + c2 * psi2[a * N3 + i];
        }
    }
}

// Full-grid index of box cell c (padded index minus the ghost width, or interior index).
__device__ __forceinline__ long long full_index(const BoxDesc &B, int Ntile, int ratio, int Ngf, int ci, int cj,
                                                int ck) {
    const long long x = wrap((B.tx * Ntile - B.Nbuf) * ratio + ci, Ngf);
    const long long y = wrap((B.ty * Ntile - B.Nbuf) * ratio + cj, Ngf);
    const long long z = wrap((B.tz * Ntile - B.Nbuf) * ratio + ck, Ngf);
    return (x * Ngf + y) * Ngf + z;
}

__global__ void __launch_bounds__(kChunk)
k_true_source(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks, const float *__restrict__ delta,
              int Ngf, int Ntile, int ratio, const float *__restrict__ phi_pad, float inv_D1, float *__restrict__ out) {
    const Chunk ch = chunks[blockIdx.x];
    const BoxDesc &B = boxes[ch.box];
    const int Ng = B.Ng;
    const long long cell = (long long)ch.start + threadIdx.x;
    if (cell >= (long long)Ng * Ng * Ng) return;
    const int k = (int)(cell % Ng), j = (int)((cell / Ng) % Ng), i = (int)(cell / Ng / Ng);
    float v = __ldg(delta + full_index(B, Ntile, ratio, Ngf, i, j, k)) * inv_D1;
    if (i < 1 || j < 1 || k < 1 || i >= Ng - 1 || j >= Ng - 1 || k >= Ng - 1) {
        const int G = B.gpad, S = Ng + 2 * G;
        const float *P = phi_pad + B.pp_off + ((i + G) * S + (j + G)) * S + (k + G);
        v -= boundary_term_n<2>(P, i, j, k, Ng, S) * (B.inv_dg * B.inv_dg);
    }
    out[B.m_off + cell] = v;
}

__global__ void __launch_bounds__(kChunk)
k_true_pad(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks, const float *__restrict__ phi,
           int Ngf, int Ntile, int ratio, float inv_D1, float *__restrict__ phi_pad) {
    const Chunk ch = chunks[blockIdx.x];
    const BoxDesc &B = boxes[ch.box];
    const long long idx = (long long)ch.start + threadIdx.x;
    if (idx >= shell_count(B.Ng, B.gpad)) return;
    int pi, pj, pk;
    shell_coord(idx, B.Ng, B.gpad, pi, pj, pk);
    const int G = B.gpad;
    const long long S = B.Ng + 2 * G;
    phi_pad[B.pp_off + ((long long)pi * S + pj) * S + pk] =
        inv_D1 * __ldg(phi + full_index(B, Ntile, ratio, Ngf, pi - G, pj - G, pk - G));
}

int grid_of(long long n, int block) {
    const long long g = (n + block - 1) / block;
    return (int)(g < 16384 ? (g > 0 ? g : 1) : 16384);
}

}  // namespace

cudaError_t launch_tc_init(Ctx &c) {
    k_tc_init<<<grid_of(c.N3, 256), 256, 0, c.stream>>>(c.tc_part, c.psi1, c.psi2, c.N3, (float)c.tt.D1_i,
                                                        (float)c.tt.D2_i);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_tc_deposit(Ctx &c) {
    const int ratio = c.tc_ng / c.Np;
    k_tc_deposit<<<grid_of(c.N3, 256), 256, 0, c.stream>>>(c.tc_part, c.N3, c.Np, c.tc_ng, (float)ratio,
                                                           (float)(c.tc_ng / c.L), c.tc_acc);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_tc_density(Ctx &c, float *delta) {
    const int ratio = c.tc_ng / c.Np;
    const float sc = (float)((double)ratio * ratio * ratio / kFix);
    k_tc_density<<<grid_of(c.tc_n3, 256), 256, 0, c.stream>>>(c.tc_acc, c.tc_n3, sc, delta);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_tc_kick_drift(Ctx &c, const float *phi, const KickDrift &kd) {
    const int ratio = c.tc_ng / c.Np;
    k_tc_kick_drift<<<(int)((c.N3 + 255) / 256), 256, 0, c.stream>>>(c.tc_part, c.psi1, c.psi2, c.N3, c.Np, c.tc_ng,
                                                                     (float)ratio, (float)(c.tc_ng / c.L), phi, kd);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_tc_final(Ctx &c, float *x, float *p) {
    const double af = c.prm.a_f;
    const double pref = af * af * c.tt.Hconf_f;
    k_tc_final<<<grid_of(c.N3, 256), 256, 0, c.stream>>>(c.tc_part, c.psi1, c.psi2, c.N3, c.Np, (float)c.dq,
                                                         (float)c.L, (float)(-pref * c.tt.dD1da_f),
                                                         (float)(pref * c.tt.dD2da_f), x, p);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_true_source(Ctx &c, const float *delta, float inv_D1) {
    if (c.n_mchunks == 0) return cudaSuccess;
    k_true_source<<<c.n_mchunks, kChunk, 0, c.stream>>>(c.boxes, c.mchunks, delta, c.tc_ng, c.Np / c.Ntiles,
                                                        c.tc_ng / c.Np, c.phi, inv_D1, c.work2);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_true_pad(Ctx &c, const float *phi, float inv_D1) {
    if (c.n_shchunks == 0) return cudaSuccess;
    k_true_pad<<<c.n_shchunks, kChunk, 0, c.stream>>>(c.boxes, c.shchunks, phi, c.tc_ng, c.Np / c.Ntiles,
                                                      c.tc_ng / c.Np, inv_D1, c.phi);
    ++c.launches;
    return cudaGetLastError();
}

}  // namespace scola
