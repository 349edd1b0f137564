// Per-box set-up and tear-down kernels (Sec. 3.2-3.3, App. B L+/L-, Sec. 4.1).
//
//  box_init   C.1-C.2 and L-: each box particle b (box-local lattice index)
//             takes the global lattice index (t Ntile - Nbuf + b) mod Np, gathers
//             Psi1, Psi2 from the full-box arrays, and starts at
//             s = -D1(a_i) Psi1 + D2(a_i) Psi2, p_res = 0 (Eqs. 39, 55).
//  shell      C.3: phi1 trilinearly interpolated (periodic, nodes at (i+1/2) d)
//             to the centre of every padded PM cell outside the interior; the
//             stencil comes from exact integer arithmetic (shell_stencil_d), the
//             weights and the eight products are formed and summed in FP64 in a
//             fixed order, and the sum is rounded once to FP32 (LEP scaling by
//             D1(a_K) happens per force evaluation, Eq. 23).  Runs once per run.
//  scatter    B.2 and L+: tile particles only; x = (q + s) mod L and
//             p = p_res + a^2 calH (-dD1/da Psi1 + dD2/da Psi2) at a_f (Eq. 55).
//  box_ids    the global id of every box particle (integer, for inspection).
//  density    periodic CIC of all particles on the N^3 LPT grid (Sec. 4.1),
//             fixed-point accumulation (deterministic), then delta = rho/nbar - 1.
#include "device_util.cuh"

namespace scola {

namespace {

__device__ __forceinline__ long long box_particle_gid(const BoxDesc &B, int Np, int Ntile, int bi,
                                                      int bj, int bk) {
    const int gi = wrap(B.tx * Ntile - B.Nbuf + bi, Np);
    const int gj = wrap(B.ty * Ntile - B.Nbuf + bj, Np);
    const int gk = wrap(B.tz * Ntile - B.Nbuf + bk, Np);
    return ((long long)gi * Np + gj) * Np + gk;
}

__global__ void __launch_bounds__(kChunk)
k_box_init(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks,
           float *__restrict__ part, long long P, const float *__restrict__ psi1,
           const float *__restrict__ psi2, int Np, int Ntile, long long N3, float D1i, float D2i) {
    const Chunk ch = chunks[blockIdx.x];
    const BoxDesc &B = boxes[ch.box];
    const int Nsc = B.Nsc;
    const int local = ch.start + threadIdx.x;
    if (local >= Nsc * Nsc * Nsc) return;
    int bi, bj, bk;
    decode_local(local, Nsc, bi, bj, bk);
    const long long gid = box_particle_gid(B, Np, Ntile, bi, bj, bk);
    const long long gi = B.p_off + local;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float q1 = psi1[a * N3 + gid];
        const float q2 = psi2[a * N3 + gid];
        part[(6 + a) * P + gi] = q1;
        part[(9 + a) * P + gi] = q2;
        part[a * P + gi] = -D1i * q1 + D2i * q2;
        part[(3 + a) * P + gi] = 0.0f;
    }
}

__global__ void __launch_bounds__(kChunk)
k_shell(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks,
        const float *__restrict__ phi1, int N, int Ntile, float *__restrict__ shell) {
    const Chunk ch = chunks[blockIdx.x];
    const BoxDesc &B = boxes[ch.box];
    const long long idx = (long long)ch.start + threadIdx.x;
    if (idx >= shell_count(B.Ng, B.gpad)) return;
    int pc[3];
    shell_coord(idx, B.Ng, B.gpad, pc[0], pc[1], pc[2]);
    int i0[3];
    double f[3];
    shell_stencil_d(B, pc, Ntile, i0, f);
    // the two periodic node indices per axis (one modulo each)
    int ix[3][2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ix[a][0] = wrap(i0[a], N);
        ix[a][1] = ix[a][0] + 1 == N ? 0 : ix[a][0] + 1;
    }
    double sum = 0.0;
    const long long NN = (long long)N * N;
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
        const double wx = dx ? f[0] : 1.0 - f[0];
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const double wxy = wx * (dy ? f[1] : 1.0 - f[1]);
            const float *row = phi1 + ix[0][dx] * NN + (long long)ix[1][dy] * N;
#pragma unroll
            for (int dz = 0; dz < 2; ++dz)
                sum = fma(wxy * (dz ? f[2] : 1.0 - f[2]), (double)row[ix[2][dz]], sum);
        }
    }
    shell[B.sh_off + idx] = (float)sum;
}

__global__ void __launch_bounds__(kChunk)
k_scatter(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks,
          const float *__restrict__ part, long long P, int Np, int Ntile, float dq, float L,
          float c1, float c2, const float *__restrict__ coefL, float *__restrict__ x, float *__restrict__ p) {
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
    const int bi = ti + B.Nbuf, bj = tj + B.Nbuf, bk = tk + B.Nbuf;
    const long long gi = B.p_off + ((long long)bi * Nsc + bj) * Nsc + bk;
    const int g[3] = {B.tx * Ntile + ti, B.ty * Ntile + tj, B.tz * Ntile + tk};
    const long long gid = ((long long)g[0] * Np + g[1]) * Np + g[2];
    const float invL = 1.0f / L;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float xv = ((float)g[a] + 0.5f) * dq + part[a * P + gi];
        xv -= L * floorf(xv * invL);
        if (xv >= L) xv -= L;
        if (xv < 0.0f) xv += L;
        x[gid * 3 + a] = xv;
        p[gid * 3 + a] = part[(3 + a) * P + gi] + c1 * part[(6 + a) * P + gi] + c2 * part[(9 + a) * P + gi];
    }
}

__global__ void __launch_bounds__(kChunk)
k_box_ids(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks, int Np, int Ntile,
          int64_t *__restrict__ out) {
    const Chunk ch = chunks[blockIdx.x];
    const BoxDesc &B = boxes[ch.box];
    const int Nsc = B.Nsc;
    const int local = ch.start + threadIdx.x;
    if (local >= Nsc * Nsc * Nsc) return;
    int bi, bj, bk;
    decode_local(local, Nsc, bi, bj, bk);
    out[B.p_off + local] = box_particle_gid(B, Np, Ntile, bi, bj, bk);
}

__global__ void k_density_deposit(const float *__restrict__ x, long long n, int N, float inv_d,
                                  unsigned long long *__restrict__ acc) {
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
        const long long NN = (long long)N * N;
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            const long long ix = wrap(i0[0] + dx, N);
            const float wx = dx ? f[0] : 1.0f - f[0];
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                const long long iy = wrap(i0[1] + dy, N);
                const float wxy = wx * (dy ? f[1] : 1.0f - f[1]);
#pragma unroll
                for (int dz = 0; dz < 2; ++dz) {
                    const long long iz = wrap(i0[2] + dz, N);
                    const float w = wxy * (dz ? f[2] : 1.0f - f[2]);
                    atomicAdd(acc + ix * NN + iy * N + iz, weight_to_fixed(w));
                }
            }
        }
    }
}

__global__ void k_density_finish(const unsigned long long *__restrict__ acc, long long n,
                                 float scale, float *__restrict__ delta) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x)
        delta[idx] = fixed_to_float(acc[idx]) * scale - 1.0f;
}

// Per box: the CIC weight its particles leave inside the interior mesh (B^sCOLA keeps it,
// Sec. 3.4.1), as 2^-32 fixed-point sums (deterministic), and the number of particles whose
// mesh coordinate lies outside [-N_ghost, Ng + N_ghost - 1] on some axis (the force
// interpolation clamps them back).  The 3D CIC weights factorise, so a particle's inside
// weight is the product over axes of its 1D weights on cells inside [0, Ng).
__global__ void __launch_bounds__(kChunk)
k_box_mass(const BoxDesc *__restrict__ boxes, const Chunk *__restrict__ chunks, const float *__restrict__ s,
           long long stride, unsigned long long *__restrict__ mass, int *__restrict__ escaped) {
    const Chunk ch = chunks[blockIdx.x];
    const BoxDesc &B = boxes[ch.box];
    const int Nsc = B.Nsc, Ng = B.Ng, ng = B.fda / 2;
    const int local = ch.start + threadIdx.x;
    unsigned long long f = 0ull;
    int out = 0;
    if (local < Nsc * Nsc * Nsc) {
        const long long gi = B.p_off + local;
        int b[3];
        decode_local(local, Nsc, b[0], b[1], b[2]);
        float w = 1.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float u_raw = fmaf(__ldg(s + a * stride + gi), B.inv_dg, fmaf((float)b[a], B.q2u, 0.5f * B.q2u - 0.5f));
            if (u_raw < -(float)ng || u_raw > (float)(Ng + ng - 1)) out = 1;
            const float u = fminf(fmaxf(u_raw, -2.0f), (float)Ng + 1.0f);
            const float fl = floorf(u);
            const int i0 = (int)fl;
            const float fr = u - fl;
            const bool in0 = (unsigned)i0 < (unsigned)Ng, in1 = (unsigned)(i0 + 1) < (unsigned)Ng;
            w *= in0 && in1 ? 1.0f : (in0 ? 1.0f - fr : (in1 ? fr : 0.0f));
        }
        f = weight_to_fixed(w);
    }
    // one atomic per warp for each sum (all lanes of a warp belong to the chunk's box)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        f += __shfl_down_sync(0xffffffffu, f, o);
        out += __shfl_down_sync(0xffffffffu, out, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (f) atomicAdd(mass + ch.box, f);
        if (out) atomicAdd(escaped + ch.box, out);
    }
}

int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    return (int)(g < 16384 ? (g > 0 ? g : 1) : 16384);
}

}  // namespace

cudaError_t launch_box_init(Ctx &c) {
    const int Ntile = c.Np / c.Ntiles;
    k_box_init<<<c.n_pchunks, kChunk, 0, c.stream>>>(c.boxes, c.pchunks, c.part, c.P, c.psi1, c.psi2,
                                                      c.Np, Ntile, c.N3, (float)c.tt.D1_i,
                                                      (float)c.tt.D2_i);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_shell(Ctx &c) {
    k_shell<<<c.n_shchunks, kChunk, 0, c.stream>>>(c.boxes, c.shchunks, c.phi1, c.Np, c.Np / c.Ntiles,
                                                    c.shell);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_scatter(Ctx &c, float *x, float *p) {
    const int Ntile = c.Np / c.Ntiles;
    const double af = c.prm.a_f;
    const double pref = af * af * c.tt.Hconf_f;
    k_scatter<<<c.n_tchunks, kChunk, 0, c.stream>>>(c.boxes, c.tchunks, c.part, c.P, c.Np, Ntile,
                                                     (float)c.dq, (float)c.L,
                                                     (float)(-pref * c.tt.dD1da_f),
                                                     (float)(pref * c.tt.dD2da_f), c.coefL, x, p);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_box_mass(Ctx &c, const float *s, unsigned long long *mass, int *escaped) {
    k_box_mass<<<c.n_pchunks, kChunk, 0, c.stream>>>(c.boxes, c.pchunks, s, c.P, mass, escaped);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_box_ids(Ctx &c, int64_t *gid) {
    k_box_ids<<<c.n_pchunks, kChunk, 0, c.stream>>>(c.boxes, c.pchunks, c.Np, c.Np / c.Ntiles, gid);
    ++c.launches;
    return cudaGetLastError();
}

cudaError_t launch_final_density(Ctx &c, const float *x, float *delta) {
    cudaError_t e = cudaMemsetAsync(c.dens_acc, 0, sizeof(unsigned long long) * c.N3, c.stream);
    if (e != cudaSuccess) return e;
    const int N = c.Np;
    k_density_deposit<<<grid_for(c.N3, 256), 256, 0, c.stream>>>(x, c.N3, N, (float)(N / c.L),
                                                                  c.dens_acc);
    ++c.launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // nbar = Np^3 / N^3 = 1 with N = Np
    k_density_finish<<<grid_for(c.N3, 256), 256, 0, c.stream>>>(c.dens_acc, c.N3,
                                                                 2.3283064365386963e-10f, delta);
    ++c.launches;
    return cudaGetLastError();
}

}  // namespace scola
