// C ABI of libscola (declared in include/scola.h): validation, device arenas,
// the full-box 2LPT stage, the per-box set-up, the captured evolution graph and
// the inspection entry points.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "device_util.cuh"

namespace scola {
namespace {
thread_local std::string g_last_error;
}
void set_error(const std::string &msg) { g_last_error = msg; }
}  // namespace scola

using namespace scola;

// Kernel classes timed in profiling mode (scola_set_profiling / scola_kernel_times).
enum KernelClass {
    KC_PAD = 0, KC_DEPOSIT, KC_DST1, KC_DST2, KC_DST3, KC_DST4, KC_DST5, KC_DST6, KC_KICK_DRIFT,
    KC_COUNT
};

struct scola_ctx : public Ctx {
    cudaStream_t cap_stream = nullptr;   // stream used only to capture the evolution graph
    long long graph_kernels = 0;         // kernels in the evolution graph
    long long lpt_kernels = 0;           // kernels of the last LPT stage
    float *w_h2d = nullptr, *x_h2d = nullptr, *p_h2d = nullptr;  // buffers of scola_forward_host
    bool profiling = false;
    std::vector<cudaEvent_t> prof_ev;    // KC_COUNT + 1 events per force evaluation
};

#define CK(call)                                                                     \
    do {                                                                             \
        cudaError_t _e = (call);                                                     \
        if (_e != cudaSuccess) {                                                     \
            set_error(std::string(#call) + ": " + cudaGetErrorString(_e));           \
            return SCOLA_ERR_CUDA;                                                   \
        }                                                                            \
    } while (0)

#define CF(call)                                                                     \
    do {                                                                             \
        cufftResult _r = (call);                                                     \
        if (_r != CUFFT_SUCCESS) {                                                   \
            set_error(std::string(#call) + ": cuFFT error " + std::to_string((int)_r)); \
            return SCOLA_ERR_CUDA;                                                   \
        }                                                                            \
    } while (0)

#define CS(call)                                                                     \
    do {                                                                             \
        scola_status _s = (call);                                                    \
        if (_s != SCOLA_OK) return _s;                                               \
    } while (0)

namespace {

constexpr bool kAutoUsesTensorCores = true;    // AUTO: three-product tensor-core form where supported
constexpr int kMaxNg = 192;  // the DST passes hold a (Ng x 32 ceil(Ng/32)) sine matrix in shared memory

struct BoxGeom {
    int nsc, ng, nbuf;
};

scola_status invalid(const std::string &m) {
    set_error(m);
    return SCOLA_ERR_INVALID_ARG;
}

// Checks the problem statement of Sec. 3.2-3.3 and computes every box's sizes.
scola_status validate(const scola_params *p, std::vector<int32_t> &bufs, std::vector<BoxGeom> &geo,
                      bool for_kernels = false) {
    if (!p) return invalid("params is NULL");
    if (!(p->L > 0)) return invalid("L must be positive");
    if (p->Np < 2) return invalid("Np must be >= 2");
    if (p->Ntiles < 1) return invalid("Ntiles must be >= 1");
    if (p->Np % p->Ntiles != 0) return invalid("Np must be a multiple of Ntiles (Sec. 3.2)");
    if (p->fda_order != 2) {
        set_error("only FDA order 2 is built");
        return SCOLA_ERR_UNSUPPORTED;
    }
    if (p->dst_variant != SCOLA_DST_SIMT && p->dst_variant != SCOLA_DST_TC_3XTF32 &&
        p->dst_variant != SCOLA_DST_TC_4XTF32 && p->dst_variant != SCOLA_DST_AUTO)
        return invalid("unknown dst_variant");
    if (p->batch_mode != SCOLA_BATCH_ALL && p->batch_mode != SCOLA_BATCH_PER_TILE)
        return invalid("unknown batch_mode");
    if (p->deposit_form != SCOLA_DEPOSIT_AUTO && p->deposit_form != SCOLA_DEPOSIT_SORTED &&
        p->deposit_form != SCOLA_DEPOSIT_ATOMIC)
        return invalid("unknown deposit_form");
    if (p->nsteps < 1) return invalid("nsteps must be >= 1");
    if (!(p->a_i > 0 && p->a_f > p->a_i)) return invalid("need 0 < a_i < a_f");
    if (!(p->Om > 0)) return invalid("Om must be positive");
    if (p->nLPT == 0) return invalid("nLPT must be non-zero");
    if (!(p->sigma8 >= 0) || !(p->h > 0)) return invalid("need sigma8 >= 0 and h > 0");
    const long long nb = (long long)p->Ntiles * p->Ntiles * p->Ntiles;
    if (nb > (1 << 20)) return invalid("too many tiles");
    bufs.assign(nb, p->Nbuf);
    if (p->buffers) {
        if (p->Ng != 0) return invalid("an explicit Ng needs uniform buffers");
        for (long long b = 0; b < nb; ++b) bufs[b] = p->buffers[b];
    }
    if (p->Ng == 0 && p->mesh_ratio < 1) return invalid("mesh_ratio must be >= 1 when Ng == 0");
    if (p->box_first < 0 || p->box_count < 0 || (long long)p->box_first + p->box_count > nb ||
        (p->box_count == 0 && p->box_first != 0))
        return invalid("box_first/box_count must select a range of boxes (or both be 0)");
    const int ntile = p->Np / p->Ntiles;
    geo.resize(nb);
    for (long long b = 0; b < nb; ++b) {
        if (bufs[b] < 0) return invalid("buffer widths must be >= 0");
        const int nsc = ntile + 2 * bufs[b];
        if (nsc > p->Np) return invalid("Np,sCOLA must not exceed Np (a box may not overlap itself)");
        const int ng = p->Ng ? p->Ng : p->mesh_ratio * nsc;
        if (ng < nsc) return invalid("Ng must be >= Np,sCOLA (Sec. 3.3, C.3)");
        if (for_kernels && ng > kMaxNg) {
            set_error("Ng > 192 is not built");
            return SCOLA_ERR_UNSUPPORTED;
        }
        if (for_kernels && (p->dst_variant == SCOLA_DST_TC_3XTF32 || p->dst_variant == SCOLA_DST_TC_4XTF32) &&
            !tc_supported(ng)) {
            set_error("the tensor-core DST needs Ng % 4 == 0 and Ng <= 128");
            return SCOLA_ERR_UNSUPPORTED;
        }
        geo[b] = {nsc, ng, bufs[b]};
    }
    return SCOLA_OK;
}

template <class T>
scola_status dev_alloc(T **ptr, long long count) {
    *ptr = nullptr;
    if (count <= 0) count = 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(ptr), sizeof(T) * (size_t)count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("cudaMalloc of ") + std::to_string(sizeof(T) * (size_t)count) +
                  " bytes: " + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SCOLA_ERR_OOM : SCOLA_ERR_CUDA;
    }
    return SCOLA_OK;
}

template <class T>
scola_status upload(T **dst, const std::vector<T> &src) {
    CS(dev_alloc(dst, (long long)src.size()));
    if (!src.empty()) CK(cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
    return SCOLA_OK;
}

void add_chunks(std::vector<Chunk> &v, int box, long long n, int per) {
    for (long long s = 0; s < n; s += per) v.push_back({box, (int)s});
}

scola_status build(scola_ctx *c, const std::vector<BoxGeom> &all_geo) {
    const scola_params &p = c->prm;
    // the boxes this context evolves: all, or the range [box_first, box_first + box_count)
    const int first = p.box_count ? p.box_first : 0;
    const int count = p.box_count ? p.box_count : (int)all_geo.size();
    const std::vector<BoxGeom> geo(all_geo.begin() + first, all_geo.begin() + first + count);
    c->Np = p.Np;
    c->Ntiles = p.Ntiles;
    c->nboxes = (int)geo.size();
    c->N3 = (long long)p.Np * p.Np * p.Np;
    c->L = p.L;
    c->dq = p.L / p.Np;
    c->tt = build_time_table(p);
    c->pk_amp = bbks_amplitude(p.Om, p.h, p.ns, p.sigma8);
    const int ntile = p.Np / p.Ntiles;

    // DST tables, one per distinct Ng
    std::map<int, int> tbl_of;
    for (const auto &g : geo) tbl_of[g.ng] = 0;
    c->max_ng = tbl_of.rbegin()->first;
    c->max_R = (c->max_ng + 31) / 32;
    const int LS = 32 * c->max_R;
    std::vector<float> arena;
    for (auto &kv : tbl_of) {
        const int Ng = kv.first;
        DstTable T;
        T.Ng = Ng;
        T.LS = LS;
        T.st_off = (long long)arena.size();
        for (int i = 0; i < Ng; ++i)
            for (int l = 0; l < LS; ++l)
                arena.push_back(l < Ng ? (float)std::sin(M_PI * (double)(l + 1) * (i + 1) / (Ng + 1))
                                       : 0.0f);
        T.lam_off = (long long)arena.size();
        kv.second = (int)c->tables_h.size();
        c->tables_h.push_back(T);
        arena.resize(arena.size() + Ng);  // eigenvalues depend on dg: filled per box below
    }
    // LPT-grid sine tables: sin(pi n/N) and sin(2 pi n/N)/d with n the wrapped wavenumber
    c->sin_half_off = (long long)arena.size();
    for (int i = 0; i < p.Np; ++i) {
        const int n = i < p.Np / 2 ? i : i - p.Np;
        arena.push_back((float)std::sin(M_PI * n / p.Np));
    }
    // colouring amplitude sqrt(P(k) / d^3) / N^3 per integer |n|^2 = nx^2 + ny^2 + nz^2 of the
    // wrapped wavenumbers (|n_i| <= N/2), from the FP64 host BBKS spectrum; entry 0 is zero
    c->amp_off = (long long)arena.size();
    {
        const double d = p.L / p.Np, kf = 2.0 * M_PI / p.L, N3 = (double)p.Np * p.Np * p.Np;
        const long long nmax = 3LL * (p.Np / 2) * (p.Np / 2);
        for (long long n2 = 0; n2 <= nmax; ++n2) {
            const double k = kf * std::sqrt((double)n2);
            const double T = bbks_transfer(k, p.Om, p.h);
            arena.push_back(n2 == 0 ? 0.0f
                                    : (float)(std::sqrt(c->pk_amp * std::pow(k, p.ns) * T * T / (d * d * d)) / N3));
        }
    }
    c->sin_full_off = (long long)arena.size();
    for (int i = 0; i < p.Np; ++i) {
        const int n = i < p.Np / 2 ? i : i - p.Np;
        arena.push_back((float)(std::sin(2.0 * M_PI * n / p.Np) / c->dq));
    }

    // boxes and work lists
    std::vector<Chunk> pch, tch, shch, zit, cit, mch, ppch;
    long long P = 0, M = 0, MP = 0, SH = 0;
    std::map<int, double> dg_of_ng;
    for (int b = 0; b < c->nboxes; ++b) {
        c->pbeg.push_back((int)pch.size());
        c->shbeg.push_back((int)shch.size());
        c->zbeg.push_back((int)zit.size());
        c->cbeg.push_back((int)cit.size());
        c->mbeg.push_back((int)mch.size());
        const BoxGeom &g = geo[b];
        BoxDesc B;
        std::memset(&B, 0, sizeof(B));
        B.Nsc = g.nsc;
        B.Ng = g.ng;
        B.Nbuf = g.nbuf;
        B.tbl = tbl_of[g.ng];
        const int gb = first + b;                      // box id in the whole tiling
        B.tx = gb / (p.Ntiles * p.Ntiles);
        B.ty = (gb / p.Ntiles) % p.Ntiles;
        B.tz = gb % p.Ntiles;
        // interior meshes start at multiples of lcm(64, Ng): aligned, and a whole number of
        // Ng-float rows from the buffer start (the tensor-core passes address them as rows)
        {
            long long q = 64;
            while (q % g.ng) q += 64;
            M = (M + q - 1) / q * q;
        }
        B.p_off = P;
        B.m_off = M;
        // padded boxes start 2 floats past a 64-float boundary: with Ng % 4 == 0 the interior
        // cells of every padded row (index 2 .. Ng+1) then start 16-byte aligned
        MP += 2;
        B.pp_off = MP;
        B.sh_off = SH;
        const double Lsc = g.nsc * c->dq;
        const double dg = Lsc / g.ng;
        B.dq = (float)c->dq;
        B.dg = (float)dg;
        B.inv_dg = (float)(1.0 / dg);
        B.q2u = (float)((double)g.ng / g.nsc);
        B.nbar_inv = (float)std::pow((double)g.ng / g.nsc, 3);
        B.dg_d = dg;
        const int t3[3] = {B.tx, B.ty, B.tz};
        for (int a = 0; a < 3; ++a) B.origin_d[a] = ((double)t3[a] * ntile - g.nbuf) * c->dq;
        c->boxes_h.push_back(B);
        const long long n = (long long)g.nsc * g.nsc * g.nsc;
        const long long ng3 = (long long)g.ng * g.ng * g.ng;
        const long long np3 = (long long)(g.ng + 4) * (g.ng + 4) * (g.ng + 4);
        add_chunks(pch, b, n, kChunk);
        add_chunks(tch, b, (long long)ntile * ntile * ntile, kChunk);
        add_chunks(shch, b, np3 - ng3, kChunk);
        add_chunks(mch, b, ng3, kChunk);
        add_chunks(ppch, b, np3, kChunk);
        const long long nz = ((long long)g.ng * g.ng + kTC - 1) / kTC;
        for (long long t = 0; t < nz; ++t) zit.push_back({b, (int)t});
        const long long nc = (long long)g.ng * ((g.ng + kTC - 1) / kTC);
        for (long long t = 0; t < nc; ++t) cit.push_back({b, (int)t});
        auto align64 = [](long long v) { return (v + 63) / 64 * 64; };
        P += n;
        M = align64(M + ng3);   // (the next box rounds up further)
        MP = align64(MP + np3);
        SH = align64(SH + np3 - ng3);
        // boxes sharing an Ng share dg only if their Np,sCOLA also matches; the
        // eigenvalue table is per Ng, so require a single dg per Ng
        auto it = dg_of_ng.find(g.ng);
        if (it == dg_of_ng.end()) {
            dg_of_ng[g.ng] = dg;
        } else if (std::fabs(it->second - dg) > 1e-12 * dg) {
            set_error("boxes with equal Ng but different Np,sCOLA are not built");
            return SCOLA_ERR_UNSUPPORTED;
        }
    }
    c->pbeg.push_back((int)pch.size());
    c->shbeg.push_back((int)shch.size());
    c->zbeg.push_back((int)zit.size());
    c->cbeg.push_back((int)cit.size());
    c->mbeg.push_back((int)mch.size());
    // deposit groups: consecutive boxes whose counts fit the L2-sized scratch (a box larger
    // than the limit forms a group of its own)
    long long dep_cells = 0;
    for (int b = 0; b < c->nboxes; ++b) {
        const long long end = c->boxes_h[b].m_off + (long long)geo[b].ng * geo[b].ng * geo[b].ng;
        if (c->dep_groups.empty() || end - c->boxes_h[c->dep_groups.back()].m_off > kDepositGroupCells)
            c->dep_groups.push_back(b);
        dep_cells = std::max(dep_cells, end - c->boxes_h[c->dep_groups.back()].m_off);
    }
    c->dep_groups.push_back(c->nboxes);
    for (auto &T : c->tables_h) {
        const double dg = dg_of_ng[T.Ng];
        for (int l = 0; l < T.Ng; ++l) {
            const double s = std::sin(M_PI * (l + 1) / (2.0 * (T.Ng + 1)));
            arena[T.lam_off + l] = (float)(-4.0 / (dg * dg) * s * s);
        }
    }
    c->P = P;
    c->M = M;
    c->MP = MP;
    c->SH = SH;
    if (pch.size() > 0x7fffffff || zit.size() > 0x7fffffff || cit.size() > 0x7fffffff)
        return invalid("problem too large for one launch");
    c->n_pchunks = (int)pch.size();
    c->n_tchunks = (int)tch.size();
    c->n_shchunks = (int)shch.size();
    c->n_zitems = (int)zit.size();
    c->n_citems = (int)cit.size();
    c->n_mchunks = (int)mch.size();
    c->n_ppchunks = (int)ppch.size();
    double r = 0;
    for (const auto &g : all_geo) r += std::pow((double)g.nsc, 3);
    c->r = r / (double)c->N3;
    c->p = (double)all_geo.size() / c->r;

    // tensor-core DST groups (one per distinct Ng): tiles and the FP32 sine matrix
    bool all_tc = true;
    for (auto &kv : tbl_of) all_tc = all_tc && tc_supported(kv.first);
    c->use_tc = (p.dst_variant == SCOLA_DST_TC_3XTF32) || (p.dst_variant == SCOLA_DST_TC_4XTF32) ||
                (p.dst_variant == SCOLA_DST_AUTO && all_tc && kAutoUsesTensorCores);
    c->tc_lo_lo = p.dst_variant == SCOLA_DST_TC_4XTF32;
    std::vector<Chunk> tct;
    std::vector<int> box_tile_beg(c->nboxes, 0), box_tile_end(c->nboxes, 0);
    if (c->use_tc) {
        for (auto &kv : tbl_of) {
            TcGroup G;
            G.Ng = kv.first;
            G.nstage = tc_plan_stages(G.Ng, G.Npad, G.nkc);
            G.lam_off = c->tables_h[kv.second].lam_off;
            G.s_off = (long long)arena.size();
            const int Kp = 32 * G.nkc;
            for (int n = 0; n < G.Npad; ++n)
                for (int k = 0; k < Kp; ++k)
                    arena.push_back(n < G.Ng && k < G.Ng
                                        ? (float)std::sin(M_PI * (double)(n + 1) * (k + 1) / (G.Ng + 1))
                                        : 0.0f);
            const long long first = (long long)tct.size();
            for (int b = 0; b < c->nboxes; ++b) {
                if (geo[b].ng != G.Ng) continue;
                const long long rows = (long long)G.Ng * G.Ng;
                box_tile_beg[b] = (int)tct.size();
                for (long long t = 0; t * kTcTileRows < rows; ++t) tct.push_back({b, (int)t});
                box_tile_end[b] = (int)tct.size();
            }
            G.ntiles = (int)(tct.size() - first);
            G.tiles = reinterpret_cast<Chunk *>(first);   // offset, rebased after upload
            c->tc_groups.push_back(G);
        }
        // per-box ranges (each box's tiles are contiguous within its group)
        c->tc_tile_beg = box_tile_beg;
        c->tc_tile_end = box_tile_end;
    }

    CK(cudaGetDevice(&c->device));
    CK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    CS(upload(&c->boxes, c->boxes_h));
    CS(upload(&c->tables, c->tables_h));
    CS(upload(&c->table_arena, arena));
    CS(upload(&c->pchunks, pch));
    CS(upload(&c->tchunks, tch));
    CS(upload(&c->shchunks, shch));
    CS(upload(&c->zitems, zit));
    CS(upload(&c->citems, cit));
    CS(upload(&c->mchunks, mch));
    CS(upload(&c->ppchunks, ppch));
    if (c->use_tc) {
        CS(upload(&c->tc_tiles, tct));
        for (auto &G : c->tc_groups) G.tiles = c->tc_tiles + reinterpret_cast<long long>(G.tiles);
        CK(init_tc_kernels());
    }
    CS(dev_alloc(&c->dev_err, 1));
    CK(cudaMemset(c->dev_err, 0, sizeof(int)));
    CS(dev_alloc(&c->part, 12 * P));
    CS(dev_alloc(&c->dep_acc, dep_cells));
    CK(cudaMemset(c->dep_acc, 0, sizeof(unsigned long long) * (size_t)dep_cells));
    CS(dev_alloc(&c->work, M));
    CS(dev_alloc(&c->work2, M));
    CS(dev_alloc(&c->phi, MP));
    CS(dev_alloc(&c->shell, SH));
    CK(cudaMemset(c->phi, 0, sizeof(float) * MP));

    const long long nc = (long long)p.Np * p.Np * (p.Np / 2 + 1);
    CS(dev_alloc(&c->ck, nc));
    CS(dev_alloc(&c->cp, nc));
    CS(dev_alloc(&c->ct, nc));
    for (int i = 0; i < 4; ++i) CS(dev_alloc(&c->g[i], c->N3));
    CS(dev_alloc(&c->phi1, c->N3));
    CS(dev_alloc(&c->phi2, c->N3));
    CS(dev_alloc(&c->psi1, 3 * c->N3));
    CS(dev_alloc(&c->psi2, 3 * c->N3));
    CS(dev_alloc(&c->dens_acc, c->N3));

    CF(cufftPlan3d(&c->plan_r2c, p.Np, p.Np, p.Np, CUFFT_R2C));
    CF(cufftPlan3d(&c->plan_c2r, p.Np, p.Np, p.Np, CUFFT_C2R));
    c->have_plans = true;
    CF(cufftSetStream(c->plan_r2c, c->stream));
    CF(cufftSetStream(c->plan_c2r, c->stream));

    CK(init_pm_kernels(*c));
    CK(init_deposit_kernels());
    for (int i = 0; i < 4; ++i) CK(cudaEventCreate(&c->ev[i]));
    CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));

    c->stats.nboxes = c->nboxes;
    c->stats.box_particles = P;
    c->stats.mesh_cells = M;
    c->stats.force_evaluations = p.nsteps + 1;
    c->stats.r = c->r;
    c->stats.p = c->p;
    return SCOLA_OK;
}

// A.1-A.2 on the full box into the context's grids.
scola_status run_lpt(scola_ctx *c, const float *w, float *delta_out) {
    const long long before = c->launches;
    const float invN3 = (float)(1.0 / (double)c->N3);
    CF(cufftExecR2C(c->plan_r2c, const_cast<cufftReal *>(reinterpret_cast<const cufftReal *>(w)), c->ck));
    CK(launch_colour(*c, c->ck));
    const size_t cbytes = sizeof(cufftComplex) * (size_t)c->Np * c->Np * (c->Np / 2 + 1);
    if (delta_out) {
        CK(cudaMemcpyAsync(c->ct, c->ck, cbytes, cudaMemcpyDeviceToDevice, c->stream));
        CF(cufftExecC2R(c->plan_c2r, c->ct, delta_out));
    }
    CK(launch_inv_laplacian(*c, c->ck, c->cp, 1.0f));
    CK(cudaMemcpyAsync(c->ct, c->cp, cbytes, cudaMemcpyDeviceToDevice, c->stream));
    CF(cufftExecC2R(c->plan_c2r, c->ct, c->phi1));
    for (int a = 0; a < 3; ++a) {
        CK(launch_second_derivative(*c, c->cp, c->ct, a, a));
        CF(cufftExecC2R(c->plan_c2r, c->ct, c->g[a]));
    }
    CK(launch_source_init(*c, c->g[0], c->g[1], c->g[2], c->g[3]));
    const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (auto &pr : pairs) {
        CK(launch_second_derivative(*c, c->cp, c->ct, pr[0], pr[1]));
        CF(cufftExecC2R(c->plan_c2r, c->ct, c->g[0]));
        CK(launch_source_sub(*c, c->g[0], c->g[3]));
    }
    CF(cufftExecR2C(c->plan_r2c, c->g[3], c->ct));
    CK(launch_inv_laplacian(*c, c->ct, c->ct, invN3));
    CF(cufftExecC2R(c->plan_c2r, c->ct, c->phi2));
    CK(launch_gradient(*c, c->phi1, c->psi1));
    CK(launch_gradient(*c, c->phi2, c->psi2));
    c->lpt_kernels = c->launches - before;
    c->lpt_done = true;
    return SCOLA_OK;
}

KickDrift kick_drift_coefficients(const TimeTable &t, int k) {
    const int n = (int)t.alpha.size();
    KickDrift kd;
    const double b = t.beta[k], D1 = t.D1[k], D2 = t.D2[k];
    kd.kF = (float)b;
    kd.k1 = (float)(-b * D1);
    kd.k2 = (float)(b * (D2 - D1 * D1));
    kd.drift = k < n;
    kd.alpha = k < n ? (float)t.alpha[k] : 0.0f;
    kd.d1 = k < n ? (float)(-t.dD1[k]) : 0.0f;
    kd.d2 = k < n ? (float)t.dD2[k] : 0.0f;
    return kd;
}

// Restricts every work list to one box; restores on destruction.
struct BoxView {
    scola_ctx *c;
    Chunk *pch, *sh, *z, *cl, *mc, *sb;
    int npch, nsh, nz, ncl, nmc, nsb;
    int view;
    BoxView(scola_ctx *cc, int b) : c(cc) {
        view = c->view_box;
        c->view_box = b;
        pch = c->pchunks; sh = c->shchunks; z = c->zitems; cl = c->citems; mc = c->mchunks; sb = c->sbricks;
        npch = c->n_pchunks; nsh = c->n_shchunks; nz = c->n_zitems; ncl = c->n_citems;
        nmc = c->n_mchunks; nsb = c->n_sbricks;
        c->sbricks = sb + c->sbbeg[b];
        c->n_sbricks = c->sbbeg[b + 1] - c->sbbeg[b];
        c->mchunks = mc + c->mbeg[b];
        c->n_mchunks = c->mbeg[b + 1] - c->mbeg[b];
        c->pchunks = pch + c->pbeg[b];
        c->n_pchunks = c->pbeg[b + 1] - c->pbeg[b];
        c->shchunks = sh + c->shbeg[b];
        c->n_shchunks = c->shbeg[b + 1] - c->shbeg[b];
        c->zitems = z + c->zbeg[b];
        c->n_zitems = c->zbeg[b + 1] - c->zbeg[b];
        c->citems = cl + c->cbeg[b];
        c->n_citems = c->cbeg[b + 1] - c->cbeg[b];
    }
    ~BoxView() {
        c->pchunks = pch; c->shchunks = sh; c->zitems = z; c->citems = cl; c->mchunks = mc; c->sbricks = sb;
        c->n_pchunks = npch; c->n_shchunks = nsh; c->n_zitems = nz; c->n_citems = ncl;
        c->n_mchunks = nmc; c->n_sbricks = nsb;
        c->view_box = view;
    }
};

// Deposit autotuner.  The deposit forms (particles sorted by brick and reduced in shared
// memory, with 256 or 512 threads per brick; or fixed-point atomics into an L2-resident
// scratch) give the same delta' bit for bit, so the choice changes only the speed.  Each
// candidate allowed by params.deposit_form is timed with CUDA events on this context's own
// boxes (one box in the per-tile form), with the particles where C.1-C.3 put them, and the
// fastest is kept for the life of the context and for its captured graph.  Runs once,
// before the first capture; needs the boxes set up (it launches C.1-C.3 itself).
scola_status autotune_deposit(scola_ctx *c) {
    if (c->tuned) return SCOLA_OK;
    struct Cand {
        int form, threads;
    };
    const Cand all[3] = {{0, 256}, {0, 512}, {1, 512}};
    int lo = 0, hi = 3;
    if (c->prm.deposit_form == SCOLA_DEPOSIT_SORTED) hi = 2;
    if (c->prm.deposit_form == SCOLA_DEPOSIT_ATOMIC) lo = 2;
    const long long launches = c->launches;
    float best = -1.0f;
    int pick = lo;
    {
        std::unique_ptr<BoxView> view;
        if (c->prm.batch_mode == SCOLA_BATCH_PER_TILE) view.reset(new BoxView(c, 0));
        CK(launch_box_init(*c));
        CK(launch_shell(*c));
        CK(launch_pad(*c, (float)c->tt.D1[0]));
        for (int q = lo; q < hi; ++q) {
            c->deposit_form = all[q].form;
            c->deposit_threads = all[q].threads;
            CK(launch_deposit(*c, c->part, c->P));          // warm-up
            float ms = -1.0f;
            for (int rep = 0; rep < 3; ++rep) {
                CK(cudaEventRecord(c->ev[3], c->stream));
                CK(launch_deposit(*c, c->part, c->P));
                CK(cudaEventRecord(c->ev[2], c->stream));
                CK(cudaEventSynchronize(c->ev[2]));
                float t = 0.0f;
                CK(cudaEventElapsedTime(&t, c->ev[3], c->ev[2]));
                if (ms < 0.0f || t < ms) ms = t;
            }
            c->stats.ms_deposit_candidates[q] = ms;
            if (best < 0.0f || ms < best) {
                best = ms;
                pick = q;
            }
        }
    }
    c->deposit_form = all[pick].form;
    c->deposit_threads = all[pick].threads;
    c->stats.deposit_form = all[pick].form == 0 ? SCOLA_DEPOSIT_SORTED : SCOLA_DEPOSIT_ATOMIC;
    c->stats.deposit_threads = all[pick].form == 0 ? all[pick].threads : 0;
    c->launches = launches;
    c->tuned = true;
    return SCOLA_OK;
}

// The plain per-tile form: every box evolved on its own, one box per launch, boxes in turn
// (the paper's one-process-per-box organisation mapped onto one GPU).
scola_status enqueue_evolution_per_tile(scola_ctx *c) {
    const int n = (int)c->tt.alpha.size();
    for (int b = 0; b < c->nboxes; ++b) {
        BoxView v(c, b);
        CK(launch_box_init(*c));
        CK(launch_shell(*c));
        for (int k = 0; k <= n; ++k) {
            CK(launch_pad(*c, (float)c->tt.D1[k]));
            CK(launch_deposit(*c, c->part, c->P));
            CK(launch_poisson(*c));
            CK(launch_kick_drift(*c, kick_drift_coefficients(c->tt, k)));
        }
    }
    return SCOLA_OK;
}

// C.1-C.3 and the whole KDK sequence on the context stream, all boxes per launch.  In
// profiling mode an external event is recorded between consecutive kernels of every
// force evaluation.
scola_status enqueue_evolution(scola_ctx *c) {
    if (c->prm.batch_mode == SCOLA_BATCH_PER_TILE) return enqueue_evolution_per_tile(c);
    CK(launch_box_init(*c));
    CK(launch_shell(*c));
    const int n = (int)c->tt.alpha.size();
    int ei = 0;
    auto mark = [&]() -> cudaError_t {
        if (!c->profiling) return cudaSuccess;
        return cudaEventRecordWithFlags(c->prof_ev[ei++], c->stream, cudaEventRecordExternal);
    };
    for (int k = 0; k <= n; ++k) {
        if (c->checkpointing)
            CK(cudaMemcpyAsync(c->ckpt + (size_t)k * 3 * c->P, c->part, sizeof(float) * 3 * (size_t)c->P,
                               cudaMemcpyDeviceToDevice, c->stream));
        CK(mark());
        CK(launch_pad(*c, (float)c->tt.D1[k]));
        CK(mark());
        CK(launch_deposit(*c, c->part, c->P));
        CK(mark());
        if (c->profiling) {
            for (int pass = 0; pass < 6; ++pass) {
                CK(launch_poisson_pass(*c, pass));
                CK(mark());
            }
        } else {
            CK(launch_poisson(*c));
        }
        CK(launch_kick_drift(*c, kick_drift_coefficients(c->tt, k)));
        CK(mark());
    }
    return SCOLA_OK;
}

scola_status ensure_graph(scola_ctx *c) {
    if (c->evolve_exec) return SCOLA_OK;
    cudaStream_t user = c->stream;
    c->stream = c->cap_stream;
    const long long before = c->launches;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    scola_status s = enqueue_evolution(c);
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    c->stream = user;
    if (s != SCOLA_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) {
        set_error(std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
        return SCOLA_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&c->evolve_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        c->evolve_exec = nullptr;
        set_error(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        return SCOLA_ERR_CUDA;
    }
    c->graph_kernels = c->launches - before;
    c->launches = before;
    return SCOLA_OK;
}

}  // namespace

extern "C" {

const char *scola_last_error(void) { return g_last_error.c_str(); }

const char *scola_status_string(scola_status s) {
    switch (s) {
        case SCOLA_OK: return "ok";
        case SCOLA_ERR_INVALID_ARG: return "invalid argument";
        case SCOLA_ERR_UNSUPPORTED: return "unsupported";
        case SCOLA_ERR_OOM: return "out of device memory";
        case SCOLA_ERR_CUDA: return "CUDA error";
        case SCOLA_ERR_STATE: return "call out of order";
        case SCOLA_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

scola_status scola_tiling_info(const scola_params *params, int32_t *box_nsc, int32_t *box_ng,
                               double *r, double *p) {
    std::vector<int32_t> bufs;
    std::vector<BoxGeom> geo;
    CS(validate(params, bufs, geo));
    double sum = 0;
    for (size_t b = 0; b < geo.size(); ++b) {
        if (box_nsc) box_nsc[b] = geo[b].nsc;
        if (box_ng) box_ng[b] = geo[b].ng;
        sum += std::pow((double)geo[b].nsc, 3);
    }
    const double rr = sum / std::pow((double)params->Np, 3);
    if (r) *r = rr;
    if (p) *p = (double)geo.size() / rr;
    return SCOLA_OK;
}

scola_status scola_time_table(const scola_params *params, double *a_force, double *D1, double *D2,
                              double *beta, double *alpha, double *dD1, double *dD2) {
    std::vector<int32_t> bufs;
    std::vector<BoxGeom> geo;
    CS(validate(params, bufs, geo));
    const TimeTable t = build_time_table(*params);
    const int n = params->nsteps;
    for (int k = 0; k <= n; ++k) {
        if (a_force) a_force[k] = t.a[k];
        if (D1) D1[k] = t.D1[k];
        if (D2) D2[k] = t.D2[k];
        if (beta) beta[k] = t.beta[k];
    }
    for (int k = 0; k < n; ++k) {
        if (alpha) alpha[k] = t.alpha[k];
        if (dD1) dD1[k] = t.dD1[k];
        if (dD2) dD2[k] = t.dD2[k];
    }
    return SCOLA_OK;
}

scola_status scola_create(const scola_params *params, void *stream, scola_ctx **out) {
    if (!out) return invalid("out is NULL");
    *out = nullptr;
    std::vector<int32_t> bufs;
    std::vector<BoxGeom> geo;
    CS(validate(params, bufs, geo, true));
    scola_ctx *c = new scola_ctx();
    c->prm = *params;
    c->prm.buffers = nullptr;
    c->buffers = bufs;
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    scola_status s = build(c, geo);
    if (s != SCOLA_OK) {
        const std::string keep = g_last_error;
        scola_destroy(c);
        set_error(keep);
        return s;
    }
    *out = c;
    return SCOLA_OK;
}

void scola_destroy(scola_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    if (c->evolve_exec) cudaGraphExecDestroy(c->evolve_exec);
    if (c->have_plans) {
        cufftDestroy(c->plan_r2c);
        cufftDestroy(c->plan_c2r);
    }
    void *ptrs[] = {c->boxes, c->tables, c->table_arena, c->pchunks, c->tchunks, c->shchunks,
                    c->zitems, c->citems, c->mchunks, c->ppchunks, c->tc_tiles, c->dev_err, c->ckpt,
                    c->adj, c->lamG, c->lam_phi_pad, c->adj_in, c->adj_out, c->lam_shell, c->lamPsi1,
                    c->lamPsi2, c->lam_phi1, c->lam_phi2, c->d2, c->lam_d2, c->part, c->dep_acc, c->kcount,
                    c->koffs, c->kcursor, c->sentries, c->sbricks,
                    c->work, c->work2, c->phi,
                    c->shell, c->ck, c->cp, c->ct, c->g[0], c->g[1], c->g[2], c->g[3], c->phi1,
                    c->phi2, c->psi1, c->psi2, c->dens_acc, c->w_h2d, c->x_h2d, c->p_h2d};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    for (auto &e : c->prof_ev)
        if (e) cudaEventDestroy(e);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

int64_t scola_box_particle_count(const scola_ctx *c) { return c ? c->P : 0; }
int64_t scola_mesh_cell_count(const scola_ctx *c) { return c ? c->M : 0; }
int64_t scola_padded_cell_count(const scola_ctx *c) { return c ? c->MP : 0; }

scola_status scola_box_offsets(const scola_ctx *c, int64_t *m_off, int64_t *pp_off, int32_t nboxes) {
    if (!c || !m_off || !pp_off) return invalid("NULL argument");
    if (nboxes != c->nboxes) return invalid("nboxes differs from the context's box count");
    for (int b = 0; b < nboxes; ++b) {
        m_off[b] = c->boxes_h[b].m_off;
        pp_off[b] = c->boxes_h[b].pp_off;
    }
    return SCOLA_OK;
}

scola_status scola_lpt_fields(scola_ctx *c, const float *w, float *delta, float *phi1, float *phi2,
                              float *psi1, float *psi2) {
    if (!c || !w) return invalid("NULL context or white noise");
    CS(run_lpt(c, w, delta));
    const size_t n = sizeof(float) * (size_t)c->N3;
    if (phi1) CK(cudaMemcpyAsync(phi1, c->phi1, n, cudaMemcpyDeviceToDevice, c->stream));
    if (phi2) CK(cudaMemcpyAsync(phi2, c->phi2, n, cudaMemcpyDeviceToDevice, c->stream));
    if (psi1) CK(cudaMemcpyAsync(psi1, c->psi1, 3 * n, cudaMemcpyDeviceToDevice, c->stream));
    if (psi2) CK(cudaMemcpyAsync(psi2, c->psi2, 3 * n, cudaMemcpyDeviceToDevice, c->stream));
    return SCOLA_OK;
}

scola_status scola_setup_boxes(scola_ctx *c) {
    if (!c) return invalid("NULL context");
    if (!c->lpt_done) {
        set_error("scola_setup_boxes needs scola_lpt_fields first");
        return SCOLA_ERR_STATE;
    }
    CS(autotune_deposit(c));
    CK(launch_box_init(*c));
    CK(launch_shell(*c));
    c->setup_done = true;
    return SCOLA_OK;
}

scola_status scola_pm_force(scola_ctx *c, const float *s, double D1, float *F, float *delta,
                            float *phi) {
    if (!c || !s || !F) return invalid("NULL argument");
    if (!c->setup_done) {
        set_error("scola_pm_force needs scola_setup_boxes first");
        return SCOLA_ERR_STATE;
    }
    CK(launch_pad(*c, (float)D1));
    CK(launch_deposit(*c, s, c->P, delta));
    CK(launch_poisson(*c));
    CK(launch_interp(*c, s, c->P, F));
    if (phi)
        CK(cudaMemcpyAsync(phi, c->phi, sizeof(float) * (size_t)c->MP, cudaMemcpyDeviceToDevice,
                           c->stream));
    return SCOLA_OK;
}

scola_status scola_box_particle_ids(scola_ctx *c, int64_t *gid) {
    if (!c || !gid) return invalid("NULL argument");
    CK(launch_box_ids(*c, gid));
    return SCOLA_OK;
}

scola_status scola_forward(scola_ctx *c, const float *w, float *x, float *p) {
    if (!c || !w || !x || !p) return invalid("NULL argument");
    const long long before = c->launches;
    CK(cudaEventRecord(c->ev[0], c->stream));
    CS(run_lpt(c, w, nullptr));
    CS(autotune_deposit(c));   // first call only; its time counts in ms_lpt
    CK(cudaEventRecord(c->ev[1], c->stream));
    CS(ensure_graph(c));
    CK(cudaGraphLaunch(c->evolve_exec, c->stream));
    CK(launch_scatter(*c, x, p));
    CK(cudaEventRecord(c->ev[2], c->stream));
    c->setup_done = true;
    c->have_forward = true;
    c->stats.kernel_launches = (c->launches - before) + c->graph_kernels;
    return SCOLA_OK;
}

scola_status scola_set_checkpointing(scola_ctx *c, int32_t enable) {
    if (!c) return invalid("NULL context");
    const bool on = enable != 0;
    if (on && c->prm.batch_mode == SCOLA_BATCH_PER_TILE) {
        set_error("the adjoint runs on the batched form only");
        return SCOLA_ERR_UNSUPPORTED;
    }
    if (on == c->checkpointing) return SCOLA_OK;
    CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    if (c->evolve_exec) {
        CK(cudaGraphExecDestroy(c->evolve_exec));
        c->evolve_exec = nullptr;
    }
    c->checkpointing = on;
    c->have_forward = false;
    if (on && !c->ckpt) {
        const long long P = c->P, N3 = c->N3;
        CS(dev_alloc(&c->ckpt, (long long)(c->prm.nsteps + 1) * 3 * P));
        CS(dev_alloc(&c->adj, 15 * P));
        CS(dev_alloc(&c->lamG, 3 * c->MP));
        CS(dev_alloc(&c->lam_phi_pad, c->MP));
        CS(dev_alloc(&c->adj_in, c->M));
        CS(dev_alloc(&c->adj_out, c->MP));
        CS(dev_alloc(&c->lam_shell, c->SH));
        CS(dev_alloc(&c->lamPsi1, 3 * N3));
        CS(dev_alloc(&c->lamPsi2, 3 * N3));
        CS(dev_alloc(&c->lam_phi1, N3));
        CS(dev_alloc(&c->lam_phi2, N3));
        CS(dev_alloc(&c->d2, 6 * N3));
        CS(dev_alloc(&c->lam_d2, 6 * N3));
    }
    return SCOLA_OK;
}

scola_status scola_backward(scola_ctx *c, const float *lam_delta, float *lam_w) {
    if (!c || !lam_delta || !lam_w) return invalid("NULL argument");
    if (!c->checkpointing || !c->have_forward) {
        set_error("scola_backward needs checkpointing enabled before the forward run it differentiates");
        return SCOLA_ERR_STATE;
    }
    const long long P = c->P, N3 = c->N3;
    const size_t fb = sizeof(float);
    CK(cudaMemsetAsync(c->adj, 0, fb * 15 * P, c->stream));
    CK(cudaMemsetAsync(c->lam_shell, 0, fb * c->SH, c->stream));
    CK(cudaMemsetAsync(c->lamPsi1, 0, fb * 3 * N3, c->stream));
    CK(cudaMemsetAsync(c->lamPsi2, 0, fb * 3 * N3, c->stream));
    CK(cudaMemsetAsync(c->lam_phi1, 0, fb * N3, c->stream));
    // final density -> tile particles
    CK(launch_adj_final(*c, lam_delta, c->adj));
    const int n = (int)c->tt.alpha.size();
    for (int k = n; k >= 0; --k) {
        CK(launch_adj_kick_drift(*c, c->adj, kick_drift_coefficients(c->tt, k)));
        const float *sk = c->ckpt + (size_t)k * 3 * P;
        CK(launch_pad(*c, (float)c->tt.D1[k]));
        CK(launch_deposit(*c, sk, P));
        CK(launch_poisson(*c));
        CK(cudaMemsetAsync(c->lamG, 0, fb * 3 * c->MP, c->stream));
        CK(launch_adj_interp(*c, sk, c->adj, c->lamG));
        CK(launch_adj_div(*c, c->lamG, c->lam_phi_pad, c->adj_in));
        CK(launch_poisson_buffers(*c, c->adj_in, c->work, c->work2, c->adj_out));
        CK(launch_adj_shell(*c, c->lam_phi_pad, c->adj_out, (float)c->tt.D1[k], c->lam_shell));
        CK(launch_adj_deposit(*c, sk, c->adj_out, c->adj));
    }
    CK(launch_adj_init_scatter(*c, c->adj, c->lamPsi1, c->lamPsi2));
    CK(launch_adj_shell_to_phi1(*c, c->lam_shell, c->lam_phi1));
    // full-box 2LPT and colouring adjoints (symmetric Fourier operators)
    CK(launch_neg_div(*c, c->lamPsi1, 1, c->lam_phi1));
    CK(launch_neg_div(*c, c->lamPsi2, 0, c->lam_phi2));
    CF(cufftExecR2C(c->plan_r2c, c->lam_phi2, c->ct));
    CK(launch_inv_laplacian(*c, c->ct, c->ct, (float)(1.0 / (double)N3)));
    CF(cufftExecC2R(c->plan_c2r, c->ct, c->g[0]));                // lam_S
    const int pairs[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    for (int q = 0; q < 6; ++q) {
        CK(launch_second_derivative(*c, c->cp, c->ct, pairs[q][0], pairs[q][1]));
        CF(cufftExecC2R(c->plan_c2r, c->ct, c->d2 + (size_t)q * N3));
    }
    CK(launch_adj_source(*c, c->g[0], c->d2, c->lam_d2));
    CF(cufftExecR2C(c->plan_r2c, c->lam_phi1, c->ck));
    for (int q = 0; q < 6; ++q) {
        CF(cufftExecR2C(c->plan_r2c, c->lam_d2 + (size_t)q * N3, c->ct));
        CK(launch_spec_d2_accumulate(*c, c->ct, c->ck, pairs[q][0], pairs[q][1]));
    }
    CK(launch_adj_colour(*c, c->ck, c->ct));
    CF(cufftExecC2R(c->plan_c2r, c->ct, lam_w));
    return SCOLA_OK;
}

scola_status scola_forward_host(scola_ctx *c, const float *w_host, float *x_host, float *p_host) {
    if (!c || !w_host || !x_host || !p_host) return invalid("NULL argument");
    if (!c->w_h2d) {
        CS(dev_alloc(&c->w_h2d, c->N3));
        CS(dev_alloc(&c->x_h2d, 3 * c->N3));
        CS(dev_alloc(&c->p_h2d, 3 * c->N3));
    }
    const size_t n = sizeof(float) * (size_t)c->N3;
    CK(cudaMemcpyAsync(c->w_h2d, w_host, n, cudaMemcpyHostToDevice, c->stream));
    CS(scola_forward(c, c->w_h2d, c->x_h2d, c->p_h2d));
    CK(cudaMemcpyAsync(x_host, c->x_h2d, 3 * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(p_host, c->p_h2d, 3 * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return SCOLA_OK;
}

scola_status scola_set_profiling(scola_ctx *c, int enable) {
    if (!c) return invalid("NULL context");
    const bool on = enable != 0;
    if (on == c->profiling) return SCOLA_OK;
    CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    if (c->evolve_exec) {
        CK(cudaGraphExecDestroy(c->evolve_exec));
        c->evolve_exec = nullptr;
    }
    c->profiling = on;
    if (on && c->prm.batch_mode == SCOLA_BATCH_PER_TILE) {
        c->profiling = false;
        set_error("profiling mode times the batched form only");
        return SCOLA_ERR_UNSUPPORTED;
    }
    if (on && c->prof_ev.empty()) {
        const size_t n = (size_t)(c->prm.nsteps + 1) * (KC_COUNT + 1);
        c->prof_ev.resize(n, nullptr);
        for (auto &e : c->prof_ev) CK(cudaEventCreate(&e));
    }
    return SCOLA_OK;
}

scola_status scola_kernel_times(const scola_ctx *cc, double *ms_per_launch, int32_t n) {
    if (!cc || !ms_per_launch) return invalid("NULL argument");
    scola_ctx *c = const_cast<scola_ctx *>(cc);
    if (!c->profiling || n < KC_COUNT) {
        set_error("scola_kernel_times needs profiling mode and room for every kernel class");
        return SCOLA_ERR_STATE;
    }
    CK(cudaEventSynchronize(c->prof_ev.back()));
    const int nf = c->prm.nsteps + 1;
    for (int q = 0; q < KC_COUNT; ++q) ms_per_launch[q] = 0.0;
    for (int k = 0; k < nf; ++k) {
        for (int q = 0; q < KC_COUNT; ++q) {
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, c->prof_ev[k * (KC_COUNT + 1) + q],
                                    c->prof_ev[k * (KC_COUNT + 1) + q + 1]));
            ms_per_launch[q] += ms / nf;
        }
    }
    return SCOLA_OK;
}

scola_status scola_device_status(scola_ctx *c) {
    if (!c) return invalid("NULL context");
    CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    int flag = 0;
    CK(cudaMemcpy(&flag, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        set_error("a kernel's bounded wait expired; its results are invalid");
        return SCOLA_ERR_TIMEOUT;
    }
    return SCOLA_OK;
}

int32_t scola_uses_tensor_cores(const scola_ctx *c) { return c && c->use_tc ? 1 : 0; }

scola_status scola_final_density(scola_ctx *c, const float *x, float *delta) {
    if (!c || !x || !delta) return invalid("NULL argument");
    CK(launch_final_density(*c, x, delta));
    return SCOLA_OK;
}

scola_status scola_get_stats(const scola_ctx *cc, scola_stats *out) {
    if (!cc || !out) return invalid("NULL argument");
    scola_ctx *c = const_cast<scola_ctx *>(cc);
    *out = c->stats;
    if (cudaEventQuery(c->ev[2]) != cudaErrorNotReady) {
        float a = 0, b = 0;
        if (cudaEventSynchronize(c->ev[2]) == cudaSuccess &&
            cudaEventElapsedTime(&a, c->ev[0], c->ev[1]) == cudaSuccess &&
            cudaEventElapsedTime(&b, c->ev[1], c->ev[2]) == cudaSuccess) {
            out->ms_lpt = a;
            out->ms_evolve = b;
        }
        cudaGetLastError();
    }
    return SCOLA_OK;
}

}  // extern "C"
