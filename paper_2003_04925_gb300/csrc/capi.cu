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
#include "fft_util.cuh"

namespace scola {
namespace {
thread_local std::string g_last_error;
thread_local std::string g_step;     // the failing step a launcher named (step_error)
}
void set_error(const std::string &msg) {
    g_last_error = g_step.empty() ? msg : msg + " [" + g_step + "]";
    g_step.clear();
}
cudaError_t step_error(const char *step, cudaError_t e) {
    g_step = step;
    return e;
}
}  // namespace scola

using namespace scola;

// Kernel classes timed in profiling mode (scola_set_profiling / scola_kernel_times).
enum KernelClass {
    KC_DEPOSIT = 0, KC_DST1, KC_DST2, KC_DST3, KC_DST4, KC_DST5, KC_DST6, KC_KICK_DRIFT,
    KC_COUNT
};

struct BoxGeom {                         // one box of the tiling: Np,sCOLA, Ng, buffer width
    int nsc, ng, nbuf;
};

struct scola_ctx : public Ctx {
    std::vector<double> a_final;         // per-tile final scale factors (empty: a_f for all)
    float *all_coef = nullptr, *all_coefL = nullptr;   // every context box's coefficients
    std::vector<BoxGeom> tiling_geo;     // every box of the tiling
    std::vector<BoxGeom> ctx_geo;        // the context's boxes
    cudaStream_t cap_stream = nullptr;   // stream used only to capture the evolution graph
    long long graph_kernels = 0;         // kernels in the evolution graph
    long long lpt_kernels = 0;           // kernels of the last LPT stage
    float *w_h2d = nullptr, *x_h2d = nullptr, *p_h2d = nullptr;  // buffers of scola_forward_host
    bool profiling = false;
    std::vector<cudaEvent_t> prof_ev;    // KC_COUNT + 1 events per force evaluation
    cudaEvent_t tc_ev[2] = {nullptr, nullptr};   // around the last periodic tCOLA run
    bool tc_timed = false;
    std::vector<cudaEvent_t> tc_prof_ev;  // profiling mode: 5 events per tCOLA force evaluation
    bool tc_profiled = false;
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

// the FP32 DST passes hold a (Ng x 32 ceil(Ng/32)) sine matrix and a column tile in shared
// memory (at most 227 KB: Ng <= 222); the tensor-core passes take Ng <= 256
constexpr int kMaxNgSimt = 222;
constexpr int kMaxNg = 256;

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
    if (p->fda_order != 2 && p->fda_order != 4 && p->fda_order != 6) {
        set_error("FDA order must be 2, 4 or 6");
        return SCOLA_ERR_UNSUPPORTED;
    }
    if (p->dst_variant != SCOLA_DST_SIMT && p->dst_variant != SCOLA_DST_TC_3XTF32 &&
        p->dst_variant != SCOLA_DST_TC_4XTF32 && p->dst_variant != SCOLA_DST_TC_3PASS &&
        p->dst_variant != SCOLA_DST_RADIX && p->dst_variant != SCOLA_DST_AUTO)
        return invalid("unknown dst_variant");
    if (p->batch_mode != SCOLA_BATCH_ALL && p->batch_mode != SCOLA_BATCH_PER_TILE)
        return invalid("unknown batch_mode");
    if (p->batch_boxes < 0) return invalid("batch_boxes must be >= 0");
    if (p->time_stepping != SCOLA_STEPPING_MODIFIED && p->time_stepping != SCOLA_STEPPING_STANDARD)
        return invalid("unknown time_stepping");
    if (p->lpt_order != 1 && p->lpt_order != 2) return invalid("lpt_order must be 1 or 2");
    if (p->study_mode < 0 || p->study_mode > 3) return invalid("study_mode must be a combination of the study flags");
    if (p->a_final) {
        const long long nt = (long long)p->Ntiles * p->Ntiles * p->Ntiles;
        for (long long t = 0; t < nt; ++t)
            if (!(p->a_final[t] > p->a_i) || !std::isfinite(p->a_final[t]))
                return invalid("every a_final must be a finite scale factor above a_i");
    }
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
        const bool tc_form = p->dst_variant == SCOLA_DST_TC_3XTF32 || p->dst_variant == SCOLA_DST_TC_4XTF32 ||
                             p->dst_variant == SCOLA_DST_TC_3PASS;
        const bool rx_form = p->dst_variant == SCOLA_DST_RADIX;
        const bool auto_form = p->dst_variant == SCOLA_DST_AUTO;
        if (for_kernels && (ng > kMaxNg || (!tc_form && !rx_form && !auto_form && ng > kMaxNgSimt))) {
            set_error("Ng > 256 is not built (Ng > 222 only with a tensor-core, radix or automatic DST form)");
            return SCOLA_ERR_UNSUPPORTED;
        }
        if (for_kernels && (rx_form || auto_form) && !rx_supported(ng) && !tc_supported(ng)) {
            set_error("the radix DST needs 1 <= Ng <= 256");
            return SCOLA_ERR_UNSUPPORTED;
        }
        if (for_kernels && tc_form && !tc_supported(ng)) {
            set_error("the tensor-core DST needs 2 <= Ng <= 240 (its sine matrix and two data stages in 227 KB of "
                      "shared memory)");
            return SCOLA_ERR_UNSUPPORTED;
        }
        geo[b] = {nsc, ng, bufs[b]};
        if (p->study_mode && ng != p->mesh_ratio * nsc) {
            set_error("the study modes need box meshes made of full-box mesh cells (Ng = mesh_ratio Np,sCOLA)");
            return SCOLA_ERR_UNSUPPORTED;
        }
    }
    if (p->study_mode && (p->fda_order != 2 || p->a_final)) {
        set_error("the study modes are built for FDA order 2 and a common final scale factor");
        return SCOLA_ERR_UNSUPPORTED;
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

// Layout of one batch of consecutive boxes [first, first + count) of the tiling: every box's
// arena offsets and, if `lists`, the work lists of every kernel and the tensor-core tiles.
// Without lists only the list lengths are counted.  Host only.
struct BatchPlan {
    std::vector<BoxGeom> geo;                          // the batch's boxes (its shape)
    std::vector<BoxDesc> boxes;
    std::vector<Chunk> pch, tch, shch, zit, cit, mch, ppch, sbr, tct;
    long long n_pch = 0, n_tch = 0, n_shch = 0, n_zit = 0, n_cit = 0, n_mch = 0, n_ppch = 0, n_sbr = 0,
              n_tct = 0;
    std::vector<int> pbeg, shbeg, zbeg, cbeg, mbeg, sbbeg, tile_beg, tile_end, dep_groups;
    std::vector<long long> group_first;                // per tensor-core group: first tile, count
    std::vector<int> group_ntiles;
    std::vector<Chunk> planes;                         // three-pass solve: (box, plane) per group
    std::vector<long long> group_plane_first;
    std::vector<int> group_nplanes, plane_beg;
    long long n_planes = 0;
    std::vector<Chunk> rxt;                            // radix DST: (box, tile) per group
    long long n_rxt = 0;
    std::vector<long long> rx_group_first;
    std::vector<int> rx_group_ntiles, rx_tile_beg, rx_tile_end;
    long long P = 0, M = 0, MP = 0, SH = 0, NK = 0, dep_cells = 0;
};

bool same_shape(const std::vector<BoxGeom> &a, const std::vector<BoxGeom> &b) {
    if (a.size() != b.size()) return false;
    for (size_t i = 0; i < a.size(); ++i)
        if (a[i].nsc != b[i].nsc || a[i].ng != b[i].ng || a[i].nbuf != b[i].nbuf) return false;
    return true;
}

void plan_batch(const scola_ctx *c, const std::vector<BoxGeom> &tiling_geo, int first, int count, bool lists,
                BatchPlan &bp) {
    const scola_params &p = c->prm;
    const int ntile = p.Np / p.Ntiles;
    bp = BatchPlan();
    bp.geo.assign(tiling_geo.begin() + first, tiling_geo.begin() + first + count);
    auto chunks = [](long long n, int per) { return (n + per - 1) / per; };
    auto add = [&](std::vector<Chunk> &v, long long &nv, int box, long long n, int per) {
        if (lists) add_chunks(v, box, n, per);
        nv += chunks(n, per);
    };
    long long P = 0, M = 0, MP = 0, SH = 0, NK = 0;
    for (int b = 0; b < count; ++b) {
        bp.pbeg.push_back((int)bp.n_pch);
        bp.shbeg.push_back((int)bp.n_shch);
        bp.zbeg.push_back((int)bp.n_zit);
        bp.cbeg.push_back((int)bp.n_cit);
        bp.mbeg.push_back((int)bp.n_mch);
        bp.sbbeg.push_back((int)bp.n_sbr);
        const BoxGeom &g = bp.geo[b];
        BoxDesc B;
        std::memset(&B, 0, sizeof(B));
        B.Nsc = g.nsc;
        B.Ng = g.ng;
        B.Nbuf = g.nbuf;
        B.tbl = c->tbl_of.at(g.ng);
        const int gb = first + b;                      // box id in the whole tiling
        B.tx = gb / (p.Ntiles * p.Ntiles);
        B.ty = (gb / p.Ntiles) % p.Ntiles;
        B.tz = gb % p.Ntiles;
        // interior meshes start at multiples of lcm(64, Ng): aligned, and a whole number of
        // Ng-float rows from the buffer start (the tensor-core passes address them as rows);
        // where the three-pass solve may run, a whole number of Ng^2-float planes (its z
        // inverse addresses the mesh as planes)
        {
            const long long unit = c->tc3_ok ? (long long)g.ng * g.ng : g.ng;
            long long q = 64;
            while (q % unit) q += 64;
            M = (M + q - 1) / q * q;
        }
        B.p_off = P;
        B.m_off = M;
        // padded boxes (G = FDA order ghost layers per side) start G mod 4 floats past a
        // 64-float boundary: with Ng % 4 == 0 the interior cells of every padded row
        // (index G .. Ng + G - 1) then start 16-byte aligned
        const int G = p.fda_order;
        MP += (G % 4 == 2) ? 2 : 0;
        B.pp_off = MP;
        B.gpad = G;
        B.fda = p.fda_order;
        B.sh_off = SH;
        {
            const int nb = (g.ng + 15) / 16;
            B.nbe = nb + 1;
            B.key_off = (int)NK;
            NK += 8LL * B.nbe * B.nbe * B.nbe;
            if (lists)
                for (int t = 0; t < nb * nb * nb; ++t) bp.sbr.push_back({b, t});
            bp.n_sbr += (long long)nb * nb * nb;
        }
        const double Lsc = g.nsc * c->dq;
        const double dg = Lsc / g.ng;
        B.dq = (float)c->dq;
        B.dg = (float)dg;
        B.inv_dg = (float)(1.0 / dg);
        B.q2u = (float)((double)g.ng / g.nsc);
        B.nbar_inv = (float)std::pow((double)g.ng / g.nsc, 3);
        B.dg_d = dg;
        B.inv_2ng_d = 1.0 / (2.0 * g.ng);
        const int t3[3] = {B.tx, B.ty, B.tz};
        for (int a = 0; a < 3; ++a) B.origin_d[a] = ((double)t3[a] * ntile - g.nbuf) * c->dq;
        bp.boxes.push_back(B);
        const long long n = (long long)g.nsc * g.nsc * g.nsc;
        const long long ng3 = (long long)g.ng * g.ng * g.ng;
        const long long np3 = (long long)(g.ng + 2 * G) * (g.ng + 2 * G) * (g.ng + 2 * G);
        add(bp.pch, bp.n_pch, b, n, kChunk);
        add(bp.tch, bp.n_tch, b, (long long)ntile * ntile * ntile, kChunk);
        add(bp.shch, bp.n_shch, b, np3 - ng3, kChunk);
        add(bp.mch, bp.n_mch, b, ng3, kChunk);
        add(bp.ppch, bp.n_ppch, b, np3, kChunk);
        const long long nz = ((long long)g.ng * g.ng + kTC - 1) / kTC;
        if (lists)
            for (long long t = 0; t < nz; ++t) bp.zit.push_back({b, (int)t});
        bp.n_zit += nz;
        const long long nc = (long long)g.ng * ((g.ng + kTC - 1) / kTC);
        if (lists)
            for (long long t = 0; t < nc; ++t) bp.cit.push_back({b, (int)t});
        bp.n_cit += nc;
        auto align64 = [](long long v) { return (v + 63) / 64 * 64; };
        P += n;
        M = align64(M + ng3);   // (the next box rounds up further)
        MP = align64(MP + np3);
        SH = align64(SH + np3 - ng3);
    }
    bp.pbeg.push_back((int)bp.n_pch);
    bp.shbeg.push_back((int)bp.n_shch);
    bp.zbeg.push_back((int)bp.n_zit);
    bp.cbeg.push_back((int)bp.n_cit);
    bp.mbeg.push_back((int)bp.n_mch);
    bp.sbbeg.push_back((int)bp.n_sbr);
    // deposit groups: consecutive boxes whose counts fit the L2-sized scratch (a box larger
    // than the limit forms a group of its own)
    for (int b = 0; b < count; ++b) {
        const long long end = bp.boxes[b].m_off + (long long)bp.geo[b].ng * bp.geo[b].ng * bp.geo[b].ng;
        if (bp.dep_groups.empty() || end - bp.boxes[bp.dep_groups.back()].m_off > kDepositGroupCells)
            bp.dep_groups.push_back(b);
        bp.dep_cells = std::max(bp.dep_cells, end - bp.boxes[bp.dep_groups.back()].m_off);
    }
    bp.dep_groups.push_back(count);
    // tensor-core DST tiles: per Ng group, each box's 256-row tiles (contiguous per box)
    bp.tile_beg.assign(count, 0);
    bp.tile_end.assign(count, 0);
    for (const TcGroup &G : c->tc_groups) {
        bp.group_first.push_back(bp.n_tct);
        for (int b = 0; b < count; ++b) {
            if (bp.geo[b].ng != G.Ng) continue;
            const long long rows = (long long)G.Ng * G.Ng;
            bp.tile_beg[b] = (int)bp.n_tct;
            for (long long t = 0; t * kTcTileRows < rows; ++t) {
                if (lists) bp.tct.push_back({b, (int)t});
                ++bp.n_tct;
            }
            bp.tile_end[b] = (int)bp.n_tct;
        }
        bp.group_ntiles.push_back((int)(bp.n_tct - bp.group_first.back()));
    }
    // plane items of the three-pass solve: per Ng group, every plane of each box
    bp.plane_beg.assign(count, 0);
    if (c->tc3_ok)
        for (const TcGroup &G : c->tc_groups) {
            bp.group_plane_first.push_back(bp.n_planes);
            for (int b = 0; b < count; ++b) {
                if (bp.geo[b].ng != G.Ng) continue;
                bp.plane_beg[b] = (int)bp.n_planes;
                for (int n = 0; n < G.Ng; ++n) {
                    if (lists) bp.planes.push_back({b, n});
                    ++bp.n_planes;
                }
            }
            bp.group_nplanes.push_back((int)(bp.n_planes - bp.group_plane_first.back()));
        }
    // radix DST tiles: per Ng group, each box's tiles of 2 R rows
    bp.rx_tile_beg.assign(count, 0);
    bp.rx_tile_end.assign(count, 0);
    for (const RxGroup &G : c->rx_groups) {
        bp.rx_group_first.push_back(bp.n_rxt);
        for (int b = 0; b < count; ++b) {
            if (bp.geo[b].ng != G.Ng) continue;
            const long long rows = (long long)G.Ng * G.Ng;
            bp.rx_tile_beg[b] = (int)bp.n_rxt;
            for (long long t = 0; t * 2 * G.R < rows; ++t) {
                if (lists) bp.rxt.push_back({b, (int)t});
                ++bp.n_rxt;
            }
            bp.rx_tile_end[b] = (int)bp.n_rxt;
        }
        bp.rx_group_ntiles.push_back((int)(bp.n_rxt - bp.rx_group_first.back()));
    }
    bp.P = P;
    bp.M = M;
    bp.MP = MP;
    bp.SH = SH;
    bp.NK = NK;
}

// Device bytes a batch of the given boxes takes in the per-batch arenas.
long long batch_bytes(const std::vector<BoxGeom> &geo, int G) {
    long long bytes = 0;
    for (const BoxGeom &g : geo) {
        const long long n = (long long)g.nsc * g.nsc * g.nsc;
        const long long ng3 = (long long)g.ng * g.ng * g.ng;
        const long long np3 = (long long)(g.ng + 2 * G) * (g.ng + 2 * G) * (g.ng + 2 * G);
        const long long nbe = (g.ng + 15) / 16 + 1;
        long long q = 64;
        while (q % g.ng) q += 64;
        bytes += 4 * 12 * n + 16 * n + 3 * 4 * 8 * nbe * nbe * nbe   // particles, sorted entries, keys
                 + 2 * 4 * (ng3 + q) + 4 * (np3 + 66) + 4 * (np3 - ng3 + 64)   // meshes, shell
                 + 8 * (2 * n / kChunk + 2 * np3 / kChunk + ng3 / kChunk + 3 * g.ng * g.ng + 64);  // lists
    }
    return bytes;
}

// Copies a host list into a preallocated device list.
template <class T>
scola_status put(T *dst, const std::vector<T> &src) {
    if (!src.empty()) CK(cudaMemcpy(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
    return SCOLA_OK;
}

// Per-tile final scale factors: the batch's boxes' coefficient tables into the fixed buffers
// the kernels (and the captured graph) read.
scola_status bind_coefficients(scola_ctx *c, int first, int count) {
    if (!c->coef) return SCOLA_OK;
    const size_t per = (size_t)c->coef_nk * 8;
    CK(cudaMemcpyAsync(c->coef, c->all_coef + (size_t)first * per, sizeof(float) * per * count,
                       cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->coefL, c->all_coefL + 2 * (size_t)first, sizeof(float) * 2 * count,
                       cudaMemcpyDeviceToDevice, c->stream));
    return SCOLA_OK;
}

// Makes batch k the one the kernels see.  A batch with the shape of the bound one only
// changes the boxes' tile coordinates (a device-to-device copy of its box descriptors,
// ordered on the stream, so the captured graph stays valid); another shape re-uploads
// the work lists (after the stream has drained) and drops the graph.
scola_status bind_batch(scola_ctx *c, int k, bool force = false) {
    if (k == c->bound_batch && !force) return SCOLA_OK;
    const int first = c->batch_first[k], count = c->batch_first[k + 1] - first;
    const BoxDesc *src = c->all_boxes + first;
    if (!force && c->bound_batch >= 0) {
        const int pf = c->batch_first[c->bound_batch];
        const int pn = c->batch_first[c->bound_batch + 1] - pf;
        std::vector<BoxGeom> a(c->ctx_geo.begin() + pf, c->ctx_geo.begin() + pf + pn);
        std::vector<BoxGeom> b(c->ctx_geo.begin() + first, c->ctx_geo.begin() + first + count);
        if (same_shape(a, b)) {
            CK(cudaMemcpyAsync(c->boxes, src, sizeof(BoxDesc) * count, cudaMemcpyDeviceToDevice, c->stream));
            CS(bind_coefficients(c, first, count));
            for (int i = 0; i < count; ++i) c->boxes_h[i] = c->all_boxes_h[first + i];
            c->bound_batch = k;
            return SCOLA_OK;
        }
    }
    BatchPlan bp;
    plan_batch(c, c->tiling_geo, c->box0 + first, count, true, bp);
    CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    if (c->evolve_exec) {
        CK(cudaGraphExecDestroy(c->evolve_exec));
        c->evolve_exec = nullptr;
    }
    CS(put(c->boxes, bp.boxes));
    CS(put(c->pchunks, bp.pch));
    CS(put(c->tchunks, bp.tch));
    CS(put(c->shchunks, bp.shch));
    CS(put(c->zitems, bp.zit));
    CS(put(c->citems, bp.cit));
    CS(put(c->mchunks, bp.mch));
    CS(put(c->ppchunks, bp.ppch));
    CS(put(c->sbricks, bp.sbr));
    if (c->use_tc) CS(put(c->tc_tiles, bp.tct));
    if (c->tc3_ok) CS(put(c->tc_planes, bp.planes));
    if (c->rx_ok) CS(put(c->rx_tiles, bp.rxt));
    c->nboxes = count;
    c->boxes_h = bp.boxes;
    c->n_pchunks = (int)bp.n_pch;
    c->n_tchunks = (int)bp.n_tch;
    c->n_shchunks = (int)bp.n_shch;
    c->n_zitems = (int)bp.n_zit;
    c->n_citems = (int)bp.n_cit;
    c->n_mchunks = (int)bp.n_mch;
    c->n_ppchunks = (int)bp.n_ppch;
    c->n_sbricks = (int)bp.n_sbr;
    c->pbeg = bp.pbeg;
    c->shbeg = bp.shbeg;
    c->zbeg = bp.zbeg;
    c->cbeg = bp.cbeg;
    c->mbeg = bp.mbeg;
    c->sbbeg = bp.sbbeg;
    c->dep_groups = bp.dep_groups;
    c->tc_tile_beg = bp.tile_beg;
    c->tc_tile_end = bp.tile_end;
    for (size_t g = 0; g < c->tc_groups.size(); ++g) {
        c->tc_groups[g].tiles = c->tc_tiles + bp.group_first[g];
        c->tc_groups[g].ntiles = bp.group_ntiles[g];
        c->tc_groups[g].planes = c->tc3_ok ? c->tc_planes + bp.group_plane_first[g] : nullptr;
        c->tc_groups[g].nplanes = c->tc3_ok ? bp.group_nplanes[g] : 0;
    }
    c->tc_plane_beg = bp.plane_beg;
    for (size_t g = 0; g < c->rx_groups.size(); ++g) {
        c->rx_groups[g].tiles = c->rx_tiles + bp.rx_group_first[g];
        c->rx_groups[g].ntiles = bp.rx_group_ntiles[g];
    }
    c->rx_tile_beg = bp.rx_tile_beg;
    c->rx_tile_end = bp.rx_tile_end;
    c->P = bp.P;
    c->M = bp.M;
    c->MP = bp.MP;
    c->SH = bp.SH;
    CS(bind_coefficients(c, first, count));
    c->bound_batch = k;
    return SCOLA_OK;
}

scola_status fill_light_cone_tables(scola_ctx *c);

// The periodic tCOLA state (once per context) and, for the study flags set, the records of
// delta_K and Phi_K at every force evaluation.
scola_status tcola_alloc(scola_ctx *c) {
    if (c->tc_part) return SCOLA_OK;
    if (c->tc_ng < 1) {
        set_error("the periodic tCOLA grid needs mesh_ratio >= 1");
        return SCOLA_ERR_UNSUPPORTED;
    }
    if (!tc_fft_supported(c->tc_ng)) {
        set_error("the periodic tCOLA grid needs 2 <= mesh_ratio Np <= 1024");
        return SCOLA_ERR_UNSUPPORTED;
    }
    CK(init_tc_fft_kernels());
    const int N = c->tc_ng;
    const long long nk = (long long)N * N * (N / 2 + 1), nrec = (long long)(c->prm.nsteps + 1) * c->tc_n3;
    CS(dev_alloc(&c->tc_acc, c->tc_n3));
    CK(cudaMemset(c->tc_acc, 0, sizeof(unsigned long long) * (size_t)c->tc_n3));
    CS(dev_alloc(&c->tc_delta, c->tc_n3));
    CS(dev_alloc(&c->tc_phi, c->tc_n3));
    CS(dev_alloc(&c->tc_dk, nk));
    CS(dev_alloc(&c->tc_dk2, nk));
    if (c->prm.study_mode & SCOLA_STUDY_TRUE_DENSITY) CS(dev_alloc(&c->rec_delta, nrec));
    if (c->prm.study_mode & SCOLA_STUDY_TRUE_POTENTIAL) CS(dev_alloc(&c->rec_phi, nrec));
    CS(dev_alloc(&c->tc_part, 6 * c->N3));
    return SCOLA_OK;
}

scola_status build(scola_ctx *c, const std::vector<BoxGeom> &all_geo) {
    const scola_params &p = c->prm;
    // the boxes this context evolves: all, or the range [box_first, box_first + box_count)
    c->box0 = p.box_count ? p.box_first : 0;
    const int count = p.box_count ? p.box_count : (int)all_geo.size();
    c->tiling_geo = all_geo;
    c->ctx_geo.assign(all_geo.begin() + c->box0, all_geo.begin() + c->box0 + count);
    const std::vector<BoxGeom> &geo = c->ctx_geo;
    c->nbox_all = count;
    c->Np = p.Np;
    c->Ntiles = p.Ntiles;
    c->N3 = (long long)p.Np * p.Np * p.Np;
    c->L = p.L;
    c->dq = p.L / p.Np;
    c->tt = build_time_table(p);
    c->pk_amp = bbks_amplitude(p.Om, p.h, p.ns, p.sigma8);

    // DST tables, one per distinct Ng
    for (const auto &g : geo) c->tbl_of[g.ng] = 0;
    c->max_ng = c->tbl_of.rbegin()->first;
    c->max_R = (c->max_ng + 31) / 32;
    const int LS = 32 * c->max_R;
    std::vector<float> arena;
    for (auto &kv : c->tbl_of) {
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
        arena.resize(arena.size() + Ng);  // eigenvalues depend on dg: filled below
    }
    // boxes sharing an Ng share dg only if their Np,sCOLA also matches; the eigenvalue
    // table is per Ng, so require a single dg per Ng
    std::map<int, double> dg_of_ng;
    for (const BoxGeom &g : geo) {
        const double dg = g.nsc * c->dq / g.ng;
        auto it = dg_of_ng.find(g.ng);
        if (it == dg_of_ng.end()) {
            dg_of_ng[g.ng] = dg;
        } else if (std::fabs(it->second - dg) > 1e-12 * dg) {
            set_error("boxes with equal Ng but different Np,sCOLA are not built");
            return SCOLA_ERR_UNSUPPORTED;
        }
    }
    for (auto &T : c->tables_h) {
        const double dg = dg_of_ng[T.Ng];
        for (int l = 0; l < T.Ng; ++l) {
            // App. C eigenvalues of the order-n second difference, t = pi l / (2 (Ng + 1))
            const double t = M_PI * (l + 1) / (2.0 * (T.Ng + 1));
            const double s1 = std::sin(t), s2 = std::sin(2 * t), s3 = std::sin(3 * t);
            double lam = -4.0 / (dg * dg) * s1 * s1;
            if (p.fda_order == 4) lam = (s2 * s2 - 16.0 * s1 * s1) / (3.0 * dg * dg);
            if (p.fda_order == 6) lam = -(2.0 * s3 * s3 - 27.0 * s2 * s2 + 270.0 * s1 * s1) / (45.0 * dg * dg);
            arena[T.lam_off + l] = (float)lam;
        }
    }
    // LPT-grid sine tables: sin(pi n/N) and sin(2 pi n/N)/d with n the wrapped wavenumber
    c->sin_half_off = (long long)arena.size();
    for (int i = 0; i < p.Np; ++i) {
        const int n = 2 * i < p.Np ? i : i - p.Np;
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
        const int n = 2 * i < p.Np ? i : i - p.Np;
        arena.push_back((float)(std::sin(2.0 * M_PI * n / p.Np) / c->dq));
    }
    // FDA order 4/6 on the LPT grid: per grid index, the 1D second-derivative symbol
    // (1/d^2)(s0 + 2 sum_m s_m cos(m k d)) and the gradient symbol (2/d) sum_m g_m sin(m k d)
    if (p.fda_order != 2) {
        static const double s4[] = {-2.5, 4.0 / 3.0, -1.0 / 12.0}, g4[] = {2.0 / 3.0, -1.0 / 12.0};
        static const double s6[] = {-49.0 / 18.0, 1.5, -0.15, 1.0 / 90.0}, g6[] = {0.75, -0.15, 1.0 / 60.0};
        const double *sc = p.fda_order == 4 ? s4 : s6, *gc = p.fda_order == 4 ? g4 : g6;
        const int ngh = p.fda_order / 2;
        const double d = c->dq;
        // (written as 2 sum_m s_m (cos(m k d) - 1), since s0 = -2 sum_m s_m: exactly 0 at k = 0)
        c->lap1_off = (long long)arena.size();
        for (int i = 0; i < p.Np; ++i) {
            const int n = 2 * i < p.Np ? i : i - p.Np;
            const double kd = 2.0 * M_PI * n / p.Np;
            double v = 0.0;
            for (int m = 1; m <= ngh; ++m) v += 2.0 * sc[m] * (std::cos(m * kd) - 1.0);
            arena.push_back((float)(v / (d * d)));
        }
        c->grad1_off = (long long)arena.size();
        for (int i = 0; i < p.Np; ++i) {
            const int n = 2 * i < p.Np ? i : i - p.Np;
            const double kd = 2.0 * M_PI * n / p.Np;
            double v = 0.0;
            for (int m = 1; m <= ngh; ++m) v += gc[m - 1] * std::sin(m * kd);
            arena.push_back((float)(2.0 * v / d));
        }
    }
    // periodic tCOLA grid (Ngf = mesh_ratio Np): the 1D FDA-2 second-derivative symbol
    // (2 / dg^2)(cos(2 pi n / Ngf) - 1) per grid index, n the wrapped wavenumber
    if (p.mesh_ratio >= 1) {
        c->tc_ng = p.mesh_ratio * p.Np;
        c->tc_n3 = (long long)c->tc_ng * c->tc_ng * c->tc_ng;
        const double dgf = p.L / c->tc_ng;
        c->tc_lap_off = (long long)arena.size();
        for (int i = 0; i < c->tc_ng; ++i) {
            const int n = 2 * i < c->tc_ng ? i : i - c->tc_ng;
            arena.push_back((float)(2.0 * (std::cos(2.0 * M_PI * n / c->tc_ng) - 1.0) / (dgf * dgf)));
        }
        // and the tables of its FFTs (twiddles; the Bluestein chirp where tc_ng is not a power of two)
        if (tc_fft_supported(c->tc_ng))
            tc_fft_tables(c->tc_ng, arena, c->tc_fft_tw_off, c->tc_fft_w_off, c->tc_fft_bk_off);
    }
    // the shared-memory FFTs' second-stage twiddles (radix DST, tCOLA Poisson solve)
    if (arena.size() & 1) arena.push_back(0.0f);
    c->fft_w256_off = (long long)arena.size();
    fft::append_w256(arena);
    // tensor-core DST groups (one per distinct Ng): the FP32 sine matrix
    bool all_tc = true;
    for (auto &kv : c->tbl_of) all_tc = all_tc && tc_supported(kv.first);
    // AUTO: the forms are set up where every Ng allows the tensor-core form, and the
    // autotuner keeps the fastest (autotune_dst); a mesh larger than the FP32 form takes
    // leaves the tensor-core form alone, one larger than the tensor-core form takes the radix
    // form
    c->dst_auto = p.dst_variant == SCOLA_DST_AUTO && all_tc && c->max_ng <= kMaxNgSimt;
    c->use_tc = (p.dst_variant == SCOLA_DST_TC_3XTF32) || (p.dst_variant == SCOLA_DST_TC_4XTF32) ||
                (p.dst_variant == SCOLA_DST_TC_3PASS) || (p.dst_variant == SCOLA_DST_AUTO && all_tc);
    c->tc_lo_lo = p.dst_variant == SCOLA_DST_TC_4XTF32;
    // the three-pass solve (plane pass, k_dst_plane.cu) where every Ng allows it
    bool all_plane = true;
    for (auto &kv : c->tbl_of) all_plane = all_plane && plane_supported(kv.first);
    c->tc3_ok = c->use_tc && all_plane && (p.dst_variant == SCOLA_DST_TC_3PASS || p.dst_variant == SCOLA_DST_AUTO);
    if (p.dst_variant == SCOLA_DST_TC_3PASS && !c->tc3_ok) {
        set_error("the three-pass tensor-core solve needs every Ng <= 96 with Ng % 4 == 0");
        return SCOLA_ERR_UNSUPPORTED;
    }
    c->tc3 = p.dst_variant == SCOLA_DST_TC_3PASS;
    // the radix form: requested, or one more autotuner candidate where every Ng allows it
    bool all_rx = true;
    for (auto &kv : c->tbl_of) all_rx = all_rx && rx_supported(kv.first);
    // (AUTO where some Ng exceeds the tensor-core form's 240: the radix form, which takes 256)
    c->rx = p.dst_variant == SCOLA_DST_RADIX || (p.dst_variant == SCOLA_DST_AUTO && !all_tc && all_rx);
    c->rx_ok = c->rx || (c->dst_auto && all_rx);
    if (c->rx_ok)
        for (auto &kv : c->tbl_of) {
            RxGroup G;
            G.Ng = kv.first;
            G.tiles = nullptr;
            G.ntiles = 0;
            G.lam_off = c->tables_h[kv.second].lam_off;
            rx_tables(G, arena);
            c->rx_groups.push_back(G);
        }
    if (c->use_tc) {
        for (auto &kv : c->tbl_of) {
            TcGroup G;
            G.Ng = kv.first;
            G.nstage = tc_plan_stages(G.Ng, G.Npad, G.nkc);
            G.nstage_zm = tc_plan_stages(G.Ng, G.Npad, G.nkc, true);
            G.planes = nullptr;
            G.nplanes = 0;
            G.lam_off = c->tables_h[kv.second].lam_off;
            G.s_off = (long long)arena.size();
            G.tiles = nullptr;
            G.ntiles = 0;
            // direct: S_nk for n, k < Ng; folded: the even-row (output 2n) and then the
            // odd-row (output 2n + 1) halves S_{2n+p, k} for n, k < ceil(Ng / 2) (even) or
            // floor(Ng / 2) (odd).  For odd Ng the even outputs' column k = (Ng - 1) / 2 (the
            // middle element, which the kernel pairs with itself: x_mid + x_mid) is halved
            const int Kp = 32 * G.nkc;
            const bool fold = tc_folded(G.Ng);
            for (int par = 0; par < (fold ? 2 : 1); ++par) {
                const int Nk = fold ? (par ? G.Ng / 2 : (G.Ng + 1) / 2) : G.Ng;
                for (int n = 0; n < G.Npad; ++n)
                    for (int k = 0; k < Kp; ++k) {
                        const int row = fold ? 2 * n + par : n;
                        const double half = (fold && par == 0 && (G.Ng & 1) && k == G.Ng / 2) ? 0.5 : 1.0;
                        arena.push_back(n < Nk && k < Nk
                                            ? (float)(half * std::sin(M_PI * (double)(row + 1) * (k + 1) / (G.Ng + 1)))
                                            : 0.0f);
                    }
            }
            c->tc_groups.push_back(G);
        }
    }
    double r = 0;
    for (const auto &g : all_geo) r += std::pow((double)g.nsc, 3);
    c->r = r / (double)c->N3;
    c->p = (double)all_geo.size() / c->r;

    CK(cudaGetDevice(&c->device));
    CK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    CS(upload(&c->tables, c->tables_h));
    CS(upload(&c->table_arena, arena));
    if (c->use_tc) CK(init_tc_kernels());
    if (c->rx_ok) CK(init_rx_kernels());
    CS(dev_alloc(&c->dev_err, 1));
    CK(cudaMemset(c->dev_err, 0, sizeof(int)));

    // full-box LPT stage (allocated first: the batches take what device memory is left)
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
    // study modes: the periodic tCOLA state and its records (before the batches are sized)
    if (p.study_mode) CS(tcola_alloc(c));

    // streamed batches: as many consecutive boxes as params.batch_boxes allows, else as fit
    // in the free device memory after a reserve for the caller's w, x, p and the host-copy
    // buffers of scola_forward_host (2 x 28 bytes per particle) and 1 GiB; the batch count
    // is then raised to a divisor of the box count where that keeps batches at least half
    // full, so that all batches share one shape (and one captured graph)
    int cap = p.batch_boxes > 0 ? p.batch_boxes : count;
    if (p.batch_boxes == 0 && count > 1) {
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        const long long reserve = 2 * 28 * c->N3 + (1LL << 30);
        const long long avail = (long long)free_b - reserve;
        long long used = 0;
        int fit = 0;
        while (fit < count) {
            const long long add = batch_bytes({geo[fit]}, p.fda_order);
            if (used + add > avail) break;
            used += add;
            ++fit;
        }
        if (fit == 0) {
            set_error("not enough device memory for one sCOLA box");
            return SCOLA_ERR_OOM;
        }
        cap = fit;
    }
    cap = std::min(cap, count);
    int nbatch = (count + cap - 1) / cap;
    for (int q = nbatch; q <= count && (count + q - 1) / q * 2 >= cap; ++q)
        if (count % q == 0) {
            nbatch = q;
            break;
        }
    const int per = (count + nbatch - 1) / nbatch;
    for (int f = 0; f < count; f += per) c->batch_first.push_back(f);
    c->batch_first.push_back(count);
    nbatch = (int)c->batch_first.size() - 1;

    // every batch's layout (box descriptors kept; list lengths and arena sizes maxed)
    long long P = 0, M = 0, MP = 0, SH = 0, NK = 0, dep = 0;
    long long L_pch = 0, L_tch = 0, L_shch = 0, L_zit = 0, L_cit = 0, L_mch = 0, L_ppch = 0, L_sbr = 0, L_tct = 0,
              L_pl = 0, L_rx = 0;
    int max_count = 0;
    for (int k = 0; k < nbatch; ++k) {
        BatchPlan bp;
        const int f = c->batch_first[k], n = c->batch_first[k + 1] - f;
        plan_batch(c, all_geo, c->box0 + f, n, false, bp);
        c->all_boxes_h.insert(c->all_boxes_h.end(), bp.boxes.begin(), bp.boxes.end());
        P = std::max(P, bp.P);
        M = std::max(M, bp.M);
        MP = std::max(MP, bp.MP);
        SH = std::max(SH, bp.SH);
        NK = std::max(NK, bp.NK);
        dep = std::max(dep, bp.dep_cells);
        L_pch = std::max(L_pch, bp.n_pch);
        L_tch = std::max(L_tch, bp.n_tch);
        L_shch = std::max(L_shch, bp.n_shch);
        L_zit = std::max(L_zit, bp.n_zit);
        L_cit = std::max(L_cit, bp.n_cit);
        L_mch = std::max(L_mch, bp.n_mch);
        L_ppch = std::max(L_ppch, bp.n_ppch);
        L_sbr = std::max(L_sbr, bp.n_sbr);
        L_tct = std::max(L_tct, bp.n_tct);
        L_pl = std::max(L_pl, bp.n_planes);
        L_rx = std::max(L_rx, bp.n_rxt);
        max_count = std::max(max_count, n);
        c->P_all += bp.P;
        for (const BoxGeom &g : bp.geo) c->M_all += (long long)g.ng * g.ng * g.ng;
    }
    const long long kInt = 0x7fffffff;
    if (L_pch > kInt || L_zit > kInt || L_cit > kInt || L_mch > kInt || L_ppch > kInt || L_shch > kInt ||
        NK > kInt || P > kInt * 4LL)
        return invalid("batch too large for one launch (set batch_boxes)");
    CS(upload(&c->all_boxes, c->all_boxes_h));
    CS(dev_alloc(&c->boxes, max_count));
    CS(dev_alloc(&c->pchunks, L_pch));
    CS(dev_alloc(&c->tchunks, L_tch));
    CS(dev_alloc(&c->shchunks, L_shch));
    CS(dev_alloc(&c->zitems, L_zit));
    CS(dev_alloc(&c->citems, L_cit));
    CS(dev_alloc(&c->mchunks, L_mch));
    CS(dev_alloc(&c->ppchunks, L_ppch));
    CS(dev_alloc(&c->sbricks, L_sbr));
    if (c->use_tc) CS(dev_alloc(&c->tc_tiles, L_tct));
    if (c->tc3_ok) CS(dev_alloc(&c->tc_planes, L_pl));
    if (c->rx_ok) CS(dev_alloc(&c->rx_tiles, L_rx));
    c->cap_P = P;
    c->cap_M = M;
    c->cap_MP = MP;
    c->cap_SH = SH;
    CS(dev_alloc(&c->part, 12 * P));
    CS(dev_alloc(&c->kcount, NK));
    CS(dev_alloc(&c->koffs, NK));
    CS(dev_alloc(&c->kcursor, NK));
    CS(dev_alloc(&c->sentries, P));
    CS(dev_alloc(&c->dep_acc, dep));
    CK(cudaMemset(c->dep_acc, 0, sizeof(unsigned long long) * (size_t)std::max(dep, 1LL)));
    CS(dev_alloc(&c->work, M));
    CS(dev_alloc(&c->work2, M));
    CS(dev_alloc(&c->phi, MP));
    CS(dev_alloc(&c->shell, SH));
    CK(cudaMemset(c->phi, 0, sizeof(float) * MP));
    if (!c->a_final.empty()) {
        CS(fill_light_cone_tables(c));
        CS(dev_alloc(&c->coef, (long long)max_count * c->coef_nk * 8));
        CS(dev_alloc(&c->coefL, 2LL * max_count));
    }
    CS(bind_batch(c, 0, true));

    if ((!c->use_tc && !c->rx) || c->dst_auto) CK(init_pm_kernels(*c));     // the FP32 DST passes
    CK(init_deposit_kernels());
    for (int i = 0; i < 4; ++i) CK(cudaEventCreate(&c->ev[i]));
    for (int i = 0; i < 2; ++i) CK(cudaEventCreate(&c->tc_ev[i]));
    CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));

    c->stats.nboxes = count;
    c->stats.box_particles = c->P_all;
    c->stats.mesh_cells = c->M_all;
    c->stats.force_evaluations = p.nsteps + 1;
    c->stats.r = c->r;
    c->stats.p = c->p;
    c->stats.batches = nbatch;
    c->stats.batch_boxes = per;
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
    CK(launch_gradient(*c, c->phi1, c->psi1));
    if (c->prm.lpt_order == 1) {
        // Zel'dovich frame: no second-order potential or displacements
        CK(cudaMemsetAsync(c->phi2, 0, sizeof(float) * (size_t)c->N3, c->stream));
        CK(cudaMemsetAsync(c->psi2, 0, sizeof(float) * 3 * (size_t)c->N3, c->stream));
        c->lpt_kernels = c->launches - before;
        c->lpt_done = true;
        return SCOLA_OK;
    }
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

// The forward kick reads the stored potential Phi / D1(a_k): its force coefficient carries
// the factor D1 (the adjoint works with Phi itself and uses kick_drift_coefficients).
KickDrift forward_kick(const TimeTable &t, int k) {
    KickDrift kd = kick_drift_coefficients(t, k);
    kd.kF = (float)(t.beta[k] * t.D1[k]);
    return kd;
}

// The periodic tCOLA run of all particles from the LPT fields of the last run_lpt, on the
// context stream.  record: keep delta_K and Phi_K of every force evaluation K for the study
// flags set (the boxes read them afterwards).
scola_status run_tcola(scola_ctx *c, bool record) {
    CS(tcola_alloc(c));
    CK(cudaEventRecord(c->tc_ev[0], c->stream));
    CK(launch_tc_init(*c));
    const int n = (int)c->tt.alpha.size();
    // profiling mode: events between the stages of every force evaluation
    const bool prof = c->profiling;
    if (prof && c->tc_prof_ev.empty()) {
        c->tc_prof_ev.assign(5 * (n + 1), nullptr);
        for (auto &e : c->tc_prof_ev) CK(cudaEventCreate(&e));
    }
    auto mark = [&](int k, int q) -> cudaError_t {
        return prof ? cudaEventRecord(c->tc_prof_ev[5 * k + q], c->stream) : cudaSuccess;
    };
    for (int k = 0; k <= n; ++k) {
        float *delta = record && c->rec_delta ? c->rec_delta + (size_t)k * c->tc_n3 : c->tc_delta;
        float *phi = record && c->rec_phi ? c->rec_phi + (size_t)k * c->tc_n3 : c->tc_phi;
        CK(mark(k, 0));
        CK(launch_tc_deposit(*c));
        CK(mark(k, 1));
        CK(launch_tc_density(*c, delta));
        CK(mark(k, 2));
        CK(launch_tc_poisson(*c, delta, phi));
        CK(mark(k, 3));
        CK(launch_tc_kick_drift(*c, phi, kick_drift_coefficients(c->tt, k)));
        CK(mark(k, 4));
    }
    c->tc_profiled = prof;
    CK(cudaEventRecord(c->tc_ev[1], c->stream));
    c->tc_timed = true;
    return SCOLA_OK;
}

// Study inputs of force evaluation k (Sec. 4.3): the ghost layers from the recorded Phi_K
// (before the source, which reads them), the Poisson source from the recorded delta_K.
// Returns whether the source was written (else the deposit makes it).
bool study_inputs(scola_ctx *c, int k, scola_status &st) {
    st = SCOLA_OK;
    const float inv_D1 = (float)(1.0 / c->tt.D1[k]);
    cudaError_t e = cudaSuccess;
    if (c->prm.study_mode & SCOLA_STUDY_TRUE_POTENTIAL)
        e = launch_true_pad(*c, c->rec_phi + (size_t)k * c->tc_n3, inv_D1);
    if (e == cudaSuccess && (c->prm.study_mode & SCOLA_STUDY_TRUE_DENSITY))
        e = launch_true_source(*c, c->rec_delta + (size_t)k * c->tc_n3, inv_D1);
    if (e != cudaSuccess) {
        set_error(std::string("study inputs: ") + cudaGetErrorString(e));
        st = SCOLA_ERR_CUDA;
    }
    return (c->prm.study_mode & SCOLA_STUDY_TRUE_DENSITY) != 0;
}

// Per-tile final scale factors: every context box's FP64 time table (one per distinct a_final)
// reduced to the FP32 coefficients the kernels read (layout in Ctx::coef).
scola_status fill_light_cone_tables(scola_ctx *c) {
    const int n = c->prm.nsteps;
    c->coef_nk = n + 1;
    std::map<double, TimeTable> tabs;
    std::vector<float> coef((size_t)c->nbox_all * c->coef_nk * 8, 0.0f), coefL(2 * (size_t)c->nbox_all);
    for (int i = 0; i < c->nbox_all; ++i) {
        const double af = c->a_final[c->box0 + i];
        auto it = tabs.find(af);
        if (it == tabs.end()) {
            scola_params q = c->prm;
            q.a_f = af;
            it = tabs.emplace(af, build_time_table(q)).first;
        }
        const TimeTable &t = it->second;
        for (int k = 0; k <= n; ++k) {
            const KickDrift kd = forward_kick(t, k);
            float *e = &coef[((size_t)i * c->coef_nk + k) * 8];
            e[0] = kd.kF;
            e[1] = kd.k1;
            e[2] = kd.k2;
            e[3] = kd.alpha;
            e[4] = kd.d1;
            e[5] = kd.d2;
            e[6] = (float)(1.0 / t.D1[k]);
            e[7] = (float)t.beta[k];          // the adjoint's kick factor (its force is Phi itself)
        }
        const double pref = af * af * t.Hconf_f;
        coefL[2 * i] = (float)(-pref * t.dD1da_f);
        coefL[2 * i + 1] = (float)(pref * t.dD2da_f);
    }
    CS(upload(&c->all_coef, coef));
    CS(upload(&c->all_coefL, coefL));
    return SCOLA_OK;
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
        int form, threads, split;
    };
    const Cand all[5] = {{0, 256, 0}, {0, 512, 0}, {0, 256, 1}, {0, 256, 2}, {1, 512, 0}};
    int lo = 0, hi = 5;
    if (c->prm.deposit_form == SCOLA_DEPOSIT_SORTED) hi = 4;
    if (c->prm.deposit_form == SCOLA_DEPOSIT_ATOMIC) lo = 4;
    const long long launches = c->launches;
    float best = -1.0f;
    int pick = lo;
    {
        std::unique_ptr<BoxView> view;
        if (c->prm.batch_mode == SCOLA_BATCH_PER_TILE) view.reset(new BoxView(c, 0));
        CK(launch_box_init(*c));
        CK(launch_shell(*c));
        CK(launch_pad(*c, 1.0f));
        const float inv_D1 = (float)(1.0 / c->tt.D1[0]);
        for (int q = lo; q < hi; ++q) {
            c->deposit_form = all[q].form;
            c->deposit_threads = all[q].threads;
            c->deposit_split = all[q].split;
            const std::string which = std::string("deposit autotuner, ") +
                                      (all[q].form == 0 ? "sorted form, " + std::to_string(all[q].threads) + " threads" +
                                                              (all[q].split == 1   ? ", 32-bit halves"
                                                               : all[q].split == 2 ? ", 16-bit halves"
                                                                                   : "")
                                                        : std::string("atomic form"));
            cudaError_t e = launch_deposit(*c, c->part, c->P, inv_D1);      // warm-up
            if (e == cudaSuccess) e = c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize();
            if (e != cudaSuccess) {
                set_error(which + ": " + cudaGetErrorString(e));
                return SCOLA_ERR_CUDA;
            }
            float ms = -1.0f;
            for (int rep = 0; rep < 3; ++rep) {
                CK(cudaEventRecord(c->ev[3], c->stream));
                CK(launch_deposit(*c, c->part, c->P, inv_D1));
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
    c->deposit_split = all[pick].split;
    c->stats.deposit_form = all[pick].form == 0 ? SCOLA_DEPOSIT_SORTED : SCOLA_DEPOSIT_ATOMIC;
    c->stats.deposit_threads = all[pick].form == 0 ? all[pick].threads : 0;
    c->stats.deposit_split = all[pick].split;
    c->launches = launches;
    c->tuned = true;
    return SCOLA_OK;
}

// Poisson-solve autotuner (SCOLA_DST_AUTO where every Ng allows the tensor-core form).  The
// candidates all meet the accuracy bound: the 3xTF32 tensor-core passes (six passes, and
// three where every Ng allows the plane pass), the dense FP32 CUDA-core passes and the radix
// (Bluestein) FP32 passes.  Each solves the context's current source (the boxes of the first
// batch, or box 0 in the per-tile form) three times after a warm-up, timed with CUDA events,
// and the fastest is kept for the life of the context and its captured graph.  Runs once,
// after autotune_deposit (whose last candidate leaves a valid source in the mesh).
scola_status autotune_dst(scola_ctx *c) {
    if (c->dst_tuned) return SCOLA_OK;
    if (!c->dst_auto) {
        c->stats.dst_form = c->rx ? SCOLA_DST_RADIX
                            : c->use_tc ? (c->tc3 ? SCOLA_DST_TC_3PASS : c->tc_lo_lo ? SCOLA_DST_TC_4XTF32
                                                                                      : SCOLA_DST_TC_3XTF32)
                                        : SCOLA_DST_SIMT;
        c->dst_tuned = true;
        return SCOLA_OK;
    }
    // candidates: tensor cores in six passes, FP32 CUDA cores, tensor cores in three passes,
    // radix FP32
    static const int forms[4] = {SCOLA_DST_TC_3XTF32, SCOLA_DST_SIMT, SCOLA_DST_TC_3PASS, SCOLA_DST_RADIX};
    static const char *names[4] = {"tensor-core form: ", "FP32 form: ", "three-pass tensor-core form: ",
                                   "radix form: "};
    auto select = [&](int q) {
        c->use_tc = q == 0 || q == 2;
        c->tc3 = q == 2;
        c->rx = q == 3;
    };
    const long long launches = c->launches;
    float t[4] = {-1.0f, -1.0f, -1.0f, -1.0f};
    {
        std::unique_ptr<BoxView> view;
        if (c->prm.batch_mode == SCOLA_BATCH_PER_TILE) view.reset(new BoxView(c, 0));
        for (int q = 0; q < 4; ++q) {
            if ((q == 2 && !c->tc3_ok) || (q == 3 && !c->rx_ok)) continue;
            select(q);
            cudaError_t e = launch_poisson(*c);
            if (e == cudaSuccess) e = c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize();
            if (e != cudaSuccess) {
                set_error(std::string("Poisson-solve autotuner, ") + names[q] + cudaGetErrorString(e));
                return SCOLA_ERR_CUDA;
            }
            for (int rep = 0; rep < 3; ++rep) {
                CK(cudaEventRecord(c->ev[3], c->stream));
                CK(launch_poisson(*c));
                CK(cudaEventRecord(c->ev[2], c->stream));
                CK(cudaEventSynchronize(c->ev[2]));
                float ms = 0.0f;
                CK(cudaEventElapsedTime(&ms, c->ev[3], c->ev[2]));
                if (t[q] < 0.0f || ms < t[q]) t[q] = ms;
            }
        }
    }
    int best = 0;
    for (int q = 1; q < 4; ++q)
        if (t[q] >= 0.0f && (t[best] < 0.0f || t[q] < t[best])) best = q;
    select(best);
    for (int q = 0; q < 4; ++q) c->stats.ms_dst_candidates[q] = t[q] < 0.0f ? 0.0 : t[q];
    c->stats.dst_form = forms[best];
    c->launches = launches;
    c->dst_tuned = true;
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
        CK(launch_pad(*c, 1.0f));
        for (int k = 0; k <= n; ++k) {
            scola_status st;
            const bool sourced = study_inputs(c, k, st);
            CS(st);
            if (!sourced) CK(launch_deposit(*c, c->part, c->P, (float)(1.0 / c->tt.D1[k]), nullptr, false, k));
            CK(launch_poisson(*c));
            CK(launch_kick_drift(*c, forward_kick(c->tt, k), false, k));
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
    CK(launch_pad(*c, 1.0f));
    const int n = (int)c->tt.alpha.size();
    int ei = 0;
    auto mark = [&]() -> cudaError_t {
        if (!c->profiling) return cudaSuccess;
        return cudaEventRecordWithFlags(c->prof_ev[ei++], c->stream, cudaEventRecordExternal);
    };
    // sorted deposit: each kick-drift counts the keys of the particles it moved, so the
    // next deposit skips its own count pass (the counts are cleared once the brick pass has
    // read them)
    const bool fused = c->deposit_form == 0 && !(c->prm.study_mode & SCOLA_STUDY_TRUE_DENSITY);
    for (int k = 0; k <= n; ++k) {
        if (c->checkpointing && k % c->ckpt_every == 0) {
            const size_t rows = c->ckpt_every == 1 ? 3 : 6;          // s, or s and p_res
            CK(cudaMemcpyAsync(c->ckpt + (size_t)(k / c->ckpt_every) * rows * c->P, c->part,
                               sizeof(float) * rows * (size_t)c->P, cudaMemcpyDeviceToDevice, c->stream));
        }
        CK(mark());
        scola_status st;
        const bool sourced = study_inputs(c, k, st);
        CS(st);
        if (!sourced) CK(launch_deposit(*c, c->part, c->P, (float)(1.0 / c->tt.D1[k]), nullptr, fused && k > 0, k));
        if (fused && k < n) CK(clear_key_counts(*c));
        CK(mark());
        if (c->profiling) {
            for (int pass = 0; pass < 6; ++pass) {
                CK(launch_poisson_pass(*c, pass));
                CK(mark());
            }
        } else {
            CK(launch_poisson(*c));
        }
        if (c->checkpointing && c->ckpt_phi && c->ckpt_every == 1)
            CK(cudaMemcpyAsync(c->ckpt_phi + (size_t)k * c->MP, c->phi, sizeof(float) * (size_t)c->MP,
                               cudaMemcpyDeviceToDevice, c->stream));
        CK(launch_kick_drift(*c, forward_kick(c->tt, k), fused, k));
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

// Checkpoint storage for the context's interval (see Ctx::ckpt_every), sized for the largest
// batch.
scola_status alloc_checkpoints(scola_ctx *c) {
    const long long P = c->cap_P;
    const int n1 = c->prm.nsteps + 1, m = c->ckpt_every;
    if (!c->ckpt) CS(dev_alloc(&c->ckpt, m == 1 ? 3LL * n1 * P : 6LL * ((n1 - 1) / m + 1) * P));
    if (m > 1 && !c->seg) CS(dev_alloc(&c->seg, 3LL * m * P));
    if (m > 1 && !c->fin) CS(dev_alloc(&c->fin, 6 * P));
    if (m == 1 && !c->ckpt_phi) {
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        const size_t need = sizeof(float) * (size_t)n1 * (size_t)c->cap_MP;
        if (need <= free_b / 2) CS(dev_alloc(&c->ckpt_phi, (long long)n1 * c->cap_MP));
    }
    c->stats.adjoint_potentials_kept = c->ckpt_phi ? 1 : 0;
    return SCOLA_OK;
}

// The per-stage and inspection entry points address one set of box arenas.
scola_status need_one_batch(const scola_ctx *c) {
    if (c->batch_first.size() == 2) return SCOLA_OK;
    set_error("this call needs a context whose boxes form one batch (set batch_boxes to the box count)");
    return SCOLA_ERR_UNSUPPORTED;
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

scola_status scola_shard_ranges(const scola_params *params, int32_t world, int32_t *first, int32_t *count) {
    std::vector<int32_t> bufs;
    std::vector<BoxGeom> geo;
    CS(validate(params, bufs, geo));
    if (!first || !count) return invalid("NULL argument");
    const int n = (int)geo.size();
    if (world < 1 || world > n) return invalid("world must be between 1 and the box count");
    // cost of a box: its particle work plus the mesh work of its Poisson solve
    std::vector<double> cost(n);
    double total = 0.0;
    for (int b = 0; b < n; ++b) {
        cost[b] = std::pow((double)geo[b].nsc, 3) + std::pow((double)geo[b].ng, 3);
        total += cost[b];
    }
    // contiguous ranges: rank r takes boxes while the running cost stays within half a box
    // of r + 1 world-th of the total, leaving at least one box for every later rank
    int start = 0;
    double acc = 0.0;
    for (int r = 0; r < world; ++r) {
        if (r == world - 1) {
            first[r] = start;
            count[r] = n - start;
            break;
        }
        const double target = total * (r + 1) / world;
        int end = start + 1;
        acc += cost[start];
        while (end < n - (world - 1 - r) && acc + cost[end] / 2.0 <= target) {
            acc += cost[end];
            ++end;
        }
        first[r] = start;
        count[r] = end - start;
        start = end;
    }
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
    if (params->a_final)
        c->a_final.assign(params->a_final, params->a_final + (long long)params->Ntiles * params->Ntiles * params->Ntiles);
    c->prm.a_final = nullptr;
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
    void *ptrs[] = {c->boxes, c->all_boxes, c->all_coef, c->all_coefL, c->coef, c->coefL, c->tables, c->table_arena, c->pchunks, c->tchunks, c->shchunks,
                    c->zitems, c->citems, c->mchunks, c->ppchunks, c->tc_tiles, c->tc_planes, c->rx_tiles, c->dev_err, c->ckpt, c->ckpt_phi, c->seg, c->fin,
                    c->adj, c->lamG, c->lam_phi_pad, c->adj_in, c->adj_out, c->lam_shell, c->lamPsi1,
                    c->lamPsi2, c->lam_phi1, c->lam_phi2, c->d2, c->lam_d2, c->part, c->dep_acc, c->kcount,
                    c->koffs, c->kcursor, c->sentries, c->sbricks,
                    c->work, c->work2, c->phi,
                    c->shell, c->ck, c->cp, c->ct, c->g[0], c->g[1], c->g[2], c->g[3], c->phi1,
                    c->phi2, c->psi1, c->psi2, c->dens_acc, c->w_h2d, c->x_h2d, c->p_h2d,
                    c->tc_part, c->tc_acc, c->tc_delta, c->tc_phi, c->tc_dk, c->tc_dk2, c->rec_delta, c->rec_phi};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    for (auto &e : c->tc_ev)
        if (e) cudaEventDestroy(e);
    for (auto &e : c->tc_prof_ev)
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
    CS(need_one_batch(c));
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
    c->have_forward = false;            // the adjoint's LPT spectra are replaced
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
    CS(need_one_batch(c));
    if (!c->lpt_done) {
        set_error("scola_setup_boxes needs scola_lpt_fields first");
        return SCOLA_ERR_STATE;
    }
    CS(autotune_deposit(c));
    CS(autotune_dst(c));
    c->have_forward = false;            // the particle state of the last forward run is replaced
    CK(launch_box_init(*c));
    CK(launch_shell(*c));
    CK(launch_pad(*c, 1.0f));
    c->setup_done = true;
    return SCOLA_OK;
}

scola_status scola_pm_force(scola_ctx *c, const float *s, double D1, float *F, float *delta,
                            float *phi) {
    if (!c || !s || !F) return invalid("NULL argument");
    CS(need_one_batch(c));
    if (!c->setup_done) {
        set_error("scola_pm_force needs scola_setup_boxes first");
        return SCOLA_ERR_STATE;
    }
    // the solve gives Phi / D1 next to the unscaled shell in the ghost layers
    CK(launch_deposit(*c, s, c->P, (float)(1.0 / D1), delta));
    CK(launch_poisson(*c));
    CK(launch_interp(*c, s, c->P, F, (float)D1));
    if (phi) CK(launch_scaled_copy(*c, c->phi, phi, c->MP, (float)D1));
    return SCOLA_OK;
}

scola_status scola_box_mass(scola_ctx *c, const float *s, double *deposited, int32_t *escaped, int32_t nboxes) {
    if (!c || !s || !deposited || !escaped) return invalid("NULL argument");
    CS(need_one_batch(c));
    if (nboxes != c->nboxes) return invalid("nboxes must be the context's box count");
    unsigned long long *mass = nullptr;
    int *esc = nullptr;
    CS(dev_alloc(&mass, nboxes));
    scola_status st = dev_alloc(&esc, nboxes);
    cudaError_t e = st == SCOLA_OK ? cudaMemsetAsync(mass, 0, sizeof(unsigned long long) * nboxes, c->stream)
                                   : cudaSuccess;
    if (st == SCOLA_OK && e == cudaSuccess) e = cudaMemsetAsync(esc, 0, sizeof(int) * nboxes, c->stream);
    if (st == SCOLA_OK && e == cudaSuccess) e = launch_box_mass(*c, s, mass, esc);
    std::vector<unsigned long long> hm(nboxes);
    std::vector<int> he(nboxes);
    if (st == SCOLA_OK && e == cudaSuccess)
        e = cudaMemcpyAsync(hm.data(), mass, sizeof(unsigned long long) * nboxes, cudaMemcpyDeviceToHost, c->stream);
    if (st == SCOLA_OK && e == cudaSuccess)
        e = cudaMemcpyAsync(he.data(), esc, sizeof(int) * nboxes, cudaMemcpyDeviceToHost, c->stream);
    if (st == SCOLA_OK && e == cudaSuccess) e = c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize();
    cudaFree(mass);
    if (esc) cudaFree(esc);
    if (st != SCOLA_OK) return st;
    if (e != cudaSuccess) {
        set_error(std::string("scola_box_mass: ") + cudaGetErrorString(e));
        return SCOLA_ERR_CUDA;
    }
    for (int b = 0; b < nboxes; ++b) {
        deposited[b] = (double)hm[b] / kFix;
        escaped[b] = he[b];
    }
    return SCOLA_OK;
}

scola_status scola_box_particle_ids(scola_ctx *c, int64_t *gid) {
    if (!c || !gid) return invalid("NULL argument");
    CS(need_one_batch(c));
    CK(launch_box_ids(*c, gid));
    return SCOLA_OK;
}

scola_status scola_forward(scola_ctx *c, const float *w, float *x, float *p) {
    if (!c || !w || !x || !p) return invalid("NULL argument");
    const long long before = c->launches;
    long long graph_kernels = 0;
    CK(cudaEventRecord(c->ev[0], c->stream));
    CS(run_lpt(c, w, nullptr));
    c->tc_timed = false;
    if (c->prm.study_mode) CS(run_tcola(c, true));   // the true delta_K and Phi_K (counts in ms_lpt)
    CS(bind_batch(c, 0));
    CS(autotune_deposit(c));   // first call only; its time counts in ms_lpt
    CS(autotune_dst(c));
    CK(cudaEventRecord(c->ev[1], c->stream));
    // the batches in turn: C.1-C.3, the evolution graph and B.2 for each
    const int nbatch = (int)c->batch_first.size() - 1;
    for (int k = 0; k < nbatch; ++k) {
        CS(bind_batch(c, k));
        CS(ensure_graph(c));
        CK(cudaGraphLaunch(c->evolve_exec, c->stream));
        graph_kernels += c->graph_kernels;
        CK(launch_scatter(*c, x, p));
    }
    CK(cudaEventRecord(c->ev[2], c->stream));
    c->setup_done = true;
    c->have_forward = true;
    c->stats.kernel_launches = (c->launches - before) + graph_kernels;
    return SCOLA_OK;
}

scola_status scola_generate_white_noise(scola_ctx *c, uint64_t seed, float *w) {
    if (!c || !w) return invalid("NULL argument");
    CK(launch_white_noise(*c, (unsigned long long)seed, w));
    return SCOLA_OK;
}

scola_status scola_tcola(scola_ctx *c, const float *w, float *x, float *p) {
    if (!c || !w || !x || !p) return invalid("NULL argument");
    if (c->prm.fda_order != 2) {
        set_error("the periodic tCOLA run is built for FDA order 2");
        return SCOLA_ERR_UNSUPPORTED;
    }
    const long long before = c->launches;
    c->have_forward = false;            // the adjoint's LPT spectra are replaced
    CS(run_lpt(c, w, nullptr));
    c->tc_timed = false;
    CS(run_tcola(c, false));
    CK(launch_tc_final(*c, x, p));
    c->stats.kernel_launches = c->launches - before;
    return SCOLA_OK;
}

scola_status scola_set_checkpointing(scola_ctx *c, int32_t enable) {
    if (!c) return invalid("NULL context");
    const bool on = enable != 0;
    if (on && c->prm.study_mode) {
        set_error("the adjoint is not built for the study modes");
        return SCOLA_ERR_UNSUPPORTED;
    }
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
    if (on) CS(alloc_checkpoints(c));
    if (on && !c->adj) {
        const long long P = c->cap_P, N3 = c->N3;
        CS(dev_alloc(&c->adj, 15 * P));
        CS(dev_alloc(&c->lamG, 4 * c->cap_MP));       // interleaved (x, y, z, unused) per padded cell
        CS(dev_alloc(&c->lam_phi_pad, c->cap_MP));
        CS(dev_alloc(&c->adj_in, c->cap_M));
        CS(dev_alloc(&c->adj_out, c->cap_MP));
        CS(dev_alloc(&c->lam_shell, c->cap_SH));
        CS(dev_alloc(&c->lamPsi1, 3 * N3));
        CS(dev_alloc(&c->lamPsi2, 3 * N3));
        CS(dev_alloc(&c->lam_phi1, N3));
        CS(dev_alloc(&c->lam_phi2, N3));
        CS(dev_alloc(&c->d2, 6 * N3));
        CS(dev_alloc(&c->lam_d2, 6 * N3));
    }
    return SCOLA_OK;
}

scola_status scola_set_checkpoint_interval(scola_ctx *c, int32_t every) {
    if (!c || every < 0) return invalid("NULL context or negative interval");
    const int n1 = c->prm.nsteps + 1;                       // force evaluations
    int m = every;
    if (m == 0) {                                           // fewest floats: slots x 6 + m x 3 (+ 6)
        long long best = -1;
        for (int q = 1; q <= n1; ++q) {
            const long long fl = q == 1 ? 3LL * n1 : 6LL * ((n1 - 1) / q + 1) + 3LL * q + 6;
            if (best < 0 || fl < best) {
                best = fl;
                m = q;
            }
        }
    }
    m = std::min(m, n1);
    if (m == c->ckpt_every) return SCOLA_OK;
    CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    if (c->evolve_exec) {                                   // the copies in the graph depend on m
        CK(cudaGraphExecDestroy(c->evolve_exec));
        c->evolve_exec = nullptr;
    }
    c->ckpt_every = m;
    c->have_forward = false;
    for (float **q : {&c->ckpt, &c->seg, &c->fin, &c->ckpt_phi})
        if (*q) {
            CK(cudaFree(*q));
            *q = nullptr;
        }
    c->stats.adjoint_potentials_kept = 0;
    if (c->checkpointing) CS(alloc_checkpoints(c));
    return SCOLA_OK;
}

int32_t scola_checkpoint_interval(const scola_ctx *c) { return c ? c->ckpt_every : 0; }

}  // extern "C"

namespace {

// The adjoint entry points need the checkpoints of a forward run made with checkpointing on,
// and no later call that replaced the LPT fields or the box state.
scola_status backward_ready(const scola_ctx *c) {
    if (!c->checkpointing || !c->have_forward) {
        set_error("the adjoint needs checkpointing enabled before the forward run it differentiates, "
                  "and no scola_lpt_fields, scola_setup_boxes or scola_tcola call after that run");
        return SCOLA_ERR_STATE;
    }
    return SCOLA_OK;
}

// Clears the full-box accumulators of the backward pass (once per call).
scola_status backward_clear_global(scola_ctx *c) {
    const long long N3 = c->N3;
    const size_t fb = sizeof(float);
    CK(cudaMemsetAsync(c->lamPsi1, 0, fb * 3 * N3, c->stream));
    CK(cudaMemsetAsync(c->lamPsi2, 0, fb * 3 * N3, c->stream));
    CK(cudaMemsetAsync(c->lam_phi1, 0, fb * N3, c->stream));
    return SCOLA_OK;
}

// Clears the bound batch's backward state; the caller then sets its tile particles' state.
scola_status backward_clear_batch(scola_ctx *c) {
    const size_t fb = sizeof(float);
    CK(cudaMemsetAsync(c->adj, 0, fb * 15 * c->P, c->stream));
    CK(cudaMemsetAsync(c->lam_shell, 0, fb * c->SH, c->stream));
    return SCOLA_OK;
}

// One force evaluation k of the reverse KDK sweep of the bound batch, with sk the box
// particles' displacements at k: the kick and drift transposes, then the mesh force
// recomputed at sk and its transpose (interpolation, gradient, Dirichlet solve, boundary
// terms, deposit).  With per-tile final scale factors every box takes its own factors of
// evaluation k from the coefficient table (k is passed on); otherwise the uniform scalars.
scola_status reverse_step(scola_ctx *c, int k, const float *sk) {
    const long long P = c->P;
    CK(launch_adj_kick_drift(*c, c->adj, kick_drift_coefficients(c->tt, k), k));
    if (c->ckpt_phi && c->ckpt_every == 1) {       // the potential the forward run kept
        CK(cudaMemcpyAsync(c->phi, c->ckpt_phi + (size_t)k * c->MP, sizeof(float) * (size_t)c->MP,
                           cudaMemcpyDeviceToDevice, c->stream));
    } else {
        CK(launch_deposit(*c, sk, P, (float)(1.0 / c->tt.D1[k]), nullptr, false, k));
        CK(launch_poisson(*c));
    }
    CK(cudaMemsetAsync(c->lamG, 0, sizeof(float) * 4 * c->MP, c->stream));
    CK(launch_adj_interp(*c, sk, c->adj, c->lamG, (float)c->tt.D1[k], k));
    CK(launch_adj_div(*c, c->lamG, c->lam_phi_pad, c->adj_in));
    CK(launch_poisson_buffers(*c, c->adj_in, c->work, c->work2, c->adj_out));
    CK(launch_adj_shell(*c, c->lam_phi_pad, c->adj_out, (float)c->tt.D1[k], c->lam_shell, k));
    CK(launch_adj_deposit(*c, sk, c->adj_out, c->adj));
    return SCOLA_OK;
}

// The reverse sweep of the bound batch from its tile particles' adjoint state in c->adj,
// accumulated into the full-box lam_Psi1, lam_Psi2 (L-) and lam_phi1 (the C.3 shell).
// Checkpoints every m-th evaluation (m > 1) hold s and p_res: each segment
// [j m, min(n, j m + m - 1)] is replayed forward from its slot (the same deterministic
// kernels, so the same displacements as the run) into seg, then swept in reverse; the
// particle arena's final state is saved before and restored after.
scola_status reverse_batch(scola_ctx *c) {
    const long long P = c->P;
    const size_t fb = sizeof(float);
    const int n = (int)c->tt.alpha.size();
    const int m = c->ckpt_every;
    if (m == 1) {
        for (int k = n; k >= 0; --k) CS(reverse_step(c, k, c->ckpt + (size_t)k * 3 * P));
    } else {
        CK(cudaMemcpyAsync(c->fin, c->part, fb * 6 * P, cudaMemcpyDeviceToDevice, c->stream));
        for (int j = n / m; j >= 0; --j) {
            const int k0 = j * m, k1 = std::min(n, k0 + m - 1);
            CK(cudaMemcpyAsync(c->part, c->ckpt + (size_t)j * 6 * P, fb * 6 * P, cudaMemcpyDeviceToDevice,
                               c->stream));
            for (int k = k0; k <= k1; ++k) {
                CK(cudaMemcpyAsync(c->seg + (size_t)(k - k0) * 3 * P, c->part, fb * 3 * P, cudaMemcpyDeviceToDevice,
                                   c->stream));
                if (k == k1) break;
                CK(launch_deposit(*c, c->part, P, (float)(1.0 / c->tt.D1[k]), nullptr, false, k));
                CK(launch_poisson(*c));
                CK(launch_kick_drift(*c, forward_kick(c->tt, k), false, k));
            }
            for (int k = k1; k >= k0; --k) CS(reverse_step(c, k, c->seg + (size_t)(k - k0) * 3 * P));
        }
        CK(cudaMemcpyAsync(c->part, c->fin, fb * 6 * P, cudaMemcpyDeviceToDevice, c->stream));
    }
    CK(launch_adj_init_scatter(*c, c->adj, c->lamPsi1, c->lamPsi2));
    CK(launch_adj_shell_to_phi1(*c, c->lam_shell, c->lam_phi1));
    return SCOLA_OK;
}

// The full-box 2LPT and colouring adjoints (symmetric Fourier operators) from the
// accumulated lam_Psi1, lam_Psi2, lam_phi1 to dLoss/dw; in the Zel'dovich frame Psi2 = 0
// does not depend on the noise and the second-order chain is absent.
scola_status lpt_adjoint(scola_ctx *c, float *lam_w) {
    const long long N3 = c->N3;
    const bool second = c->prm.lpt_order == 2;
    CK(launch_neg_div(*c, c->lamPsi1, 1, c->lam_phi1));
    const int pairs[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    if (second) {
        CK(launch_neg_div(*c, c->lamPsi2, 0, c->lam_phi2));
        CF(cufftExecR2C(c->plan_r2c, c->lam_phi2, c->ct));
        CK(launch_inv_laplacian(*c, c->ct, c->ct, (float)(1.0 / (double)N3)));
        CF(cufftExecC2R(c->plan_c2r, c->ct, c->g[0]));                // lam_S
        for (int q = 0; q < 6; ++q) {
            CK(launch_second_derivative(*c, c->cp, c->ct, pairs[q][0], pairs[q][1]));
            CF(cufftExecC2R(c->plan_c2r, c->ct, c->d2 + (size_t)q * N3));
        }
        CK(launch_adj_source(*c, c->g[0], c->d2, c->lam_d2));
    }
    CF(cufftExecR2C(c->plan_r2c, c->lam_phi1, c->ck));
    for (int q = 0; second && q < 6; ++q) {
        CF(cufftExecR2C(c->plan_r2c, c->lam_d2 + (size_t)q * N3, c->ct));
        CK(launch_spec_d2_accumulate(*c, c->ct, c->ck, pairs[q][0], pairs[q][1]));
    }
    CK(launch_adj_colour(*c, c->ck, c->ct));
    CF(cufftExecC2R(c->plan_c2r, c->ct, lam_w));
    return SCOLA_OK;
}

// The whole backward pass.  One batch: its checkpoints are those of the forward run.  Several
// streamed batches: each batch is bound in turn and its evolution replayed from C.1 with the
// checkpointing graph (deterministic: the run's own trajectory, and its checkpoints), its
// tile particles take their initial adjoint state (init), and its reverse sweep accumulates
// into the full-box arrays; the LPT and colouring adjoints run once at the end.
template <typename Init>
scola_status backward_all(scola_ctx *c, float *lam_w, Init init) {
    CS(backward_clear_global(c));
    const int nbatch = (int)c->batch_first.size() - 1;
    for (int b = 0; b < nbatch; ++b) {
        if (nbatch > 1) {
            CS(bind_batch(c, b));
            CS(ensure_graph(c));
            CK(cudaGraphLaunch(c->evolve_exec, c->stream));
        }
        CS(backward_clear_batch(c));
        CK(init());
        CS(reverse_batch(c));
    }
    return lpt_adjoint(c, lam_w);
}

}  // namespace

extern "C" {

scola_status scola_backward(scola_ctx *c, const float *lam_x, const float *lam_p, float *lam_w) {
    if (!c || !lam_w || (!lam_x && !lam_p)) return invalid("NULL argument (lam_w, or both lam_x and lam_p)");
    CS(backward_ready(c));
    return backward_all(c, lam_w, [&]() { return launch_adj_final_xp(*c, lam_x, lam_p, c->adj); });
}

scola_status scola_backward_density(scola_ctx *c, const float *lam_delta, float *lam_w) {
    if (!c || !lam_delta || !lam_w) return invalid("NULL argument");
    CS(backward_ready(c));
    // final density -> tile particles (from the batch's final particle state)
    return backward_all(c, lam_w, [&]() { return launch_adj_final(*c, lam_delta, c->adj); });
}

scola_status scola_density_adjoint(scola_ctx *c, const float *x, const float *lam_delta, float *lam_x) {
    if (!c || !x || !lam_delta || !lam_x) return invalid("NULL argument");
    CK(launch_density_vjp(*c, x, lam_delta, lam_x));
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

scola_status scola_tcola_kernel_times(const scola_ctx *cc, double *ms_per_launch, int32_t n) {
    if (!cc || !ms_per_launch) return invalid("NULL argument");
    scola_ctx *c = const_cast<scola_ctx *>(cc);
    if (!c->tc_profiled || n < 4) {
        set_error("scola_tcola_kernel_times needs a tCOLA run made in profiling mode and room for 4 stages");
        return SCOLA_ERR_STATE;
    }
    CK(cudaEventSynchronize(c->tc_prof_ev.back()));
    const int nf = c->prm.nsteps + 1;
    for (int q = 0; q < 4; ++q) ms_per_launch[q] = 0.0;
    for (int k = 0; k < nf; ++k)
        for (int q = 0; q < 4; ++q) {
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, c->tc_prof_ev[5 * k + q], c->tc_prof_ev[5 * k + q + 1]));
            ms_per_launch[q] += ms / nf;
        }
    return SCOLA_OK;
}

scola_status scola_device_status(scola_ctx *c) {
    if (!c) return invalid("NULL context");
    CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    int flag = 0;
    CK(cudaMemcpy(&flag, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) CK(cudaMemset(c->dev_err, 0, sizeof(int)));     // reported once
    if (flag & 1) {
        set_error("a kernel's bounded wait expired; its results are invalid");
        return SCOLA_ERR_TIMEOUT;
    }
    if (flag & 2) {
        set_error("sorted deposit: a fill pass found more particles for a key than its count pass "
                  "(nothing was written past the slice); the densities are invalid");
        return SCOLA_ERR_CUDA;
    }
    return SCOLA_OK;
}

scola_status scola_selftest_wait_timeout(scola_ctx *c, double wait_seconds) {
    if (!c || !(wait_seconds > 0.0) || wait_seconds > 2.0) return invalid("NULL context or wait outside (0, 2] s");
    CS(need_one_batch(c));
    if (!c->use_tc) {
        set_error("the context does not use the tensor-core DST");
        return SCOLA_ERR_UNSUPPORTED;
    }
    if (!c->setup_done) {
        set_error("scola_selftest_wait_timeout needs a forward run or scola_setup_boxes first");
        return SCOLA_ERR_STATE;
    }
    CS(scola_device_status(c));                                // nothing pending before the test
    c->tc_stall_ns = (unsigned long long)(wait_seconds * 1e9);
    const cudaError_t e = launch_poisson_tc_pass(*c, 0);       // work2 -> work: scratch meshes only
    c->tc_stall_ns = 0;
    CK(e);
    return scola_device_status(c);
}

int32_t scola_uses_tensor_cores(const scola_ctx *c) { return c && c->use_tc ? 1 : 0; }

scola_status scola_final_density(scola_ctx *c, const float *x, float *delta) {
    if (!c || !x || !delta) return invalid("NULL argument");
    CK(launch_final_density(*c, x, delta));
    return SCOLA_OK;
}

scola_status scola_power_spectrum(scola_ctx *c, const float *delta, int32_t nbins, const double *edges,
                                  double *k_mean, double *pk, int64_t *n_modes) {
    if (!c || !delta || !edges || !k_mean || !pk || !n_modes) return invalid("NULL argument");
    if (nbins < 1 || nbins > kMaxSpectrumBins) return invalid("nbins must be in [1, 2048]");
    for (int b = 0; b < nbins; ++b)
        if (!(edges[b] < edges[b + 1])) return invalid("bin edges must increase");
    // the bin of each integer n^2 = |n|^2 of the wrapped wavenumbers, from k = kf sqrt(n^2)
    // in FP64: bin b holds edges[b] <= k < edges[b + 1]
    const int N = c->Np;
    const long long nmax = 3LL * (N / 2) * (N / 2);
    const double kf = 2.0 * M_PI / c->L;
    std::vector<int> bin(nmax + 1);
    for (long long n2 = 0; n2 <= nmax; ++n2) {
        const double k = kf * std::sqrt((double)n2);
        const int b = (int)(std::upper_bound(edges, edges + nbins + 1, k) - edges) - 1;
        bin[n2] = (b >= 0 && b < nbins) ? b : -1;
    }
    const int rows = 2 * c->num_sms;
    int *bin_d = nullptr;
    double *scratch = nullptr, *out_d = nullptr;
    scola_status st = upload(&bin_d, bin);
    if (st == SCOLA_OK) st = dev_alloc(&scratch, 3LL * rows * nbins);
    if (st == SCOLA_OK) st = dev_alloc(&out_d, 3LL * nbins);
    std::vector<double> out(3 * (size_t)nbins);
    cudaError_t e = cudaSuccess;
    cufftResult fr = CUFFT_SUCCESS;
    if (st == SCOLA_OK) {
        // transform a copy (the grid scratch g[0]): the caller's field stays untouched
        e = cudaMemcpyAsync(c->g[0], delta, sizeof(float) * (size_t)c->N3, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) fr = cufftExecR2C(c->plan_r2c, c->g[0], c->ck);
        if (e == cudaSuccess && fr == CUFFT_SUCCESS) e = launch_spectrum(*c, c->ck, bin_d, nbins, scratch, rows, out_d);
        if (e == cudaSuccess && fr == CUFFT_SUCCESS)
            e = cudaMemcpyAsync(out.data(), out_d, sizeof(double) * out.size(), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && fr == CUFFT_SUCCESS) e = cudaStreamSynchronize(c->stream);
    }
    cudaFree(bin_d);
    cudaFree(scratch);
    cudaFree(out_d);
    if (st != SCOLA_OK) return st;
    if (fr != CUFFT_SUCCESS) {
        set_error("cufftExecR2C: cuFFT error " + std::to_string((int)fr));
        return SCOLA_ERR_CUDA;
    }
    CK(e);
    const double norm = std::pow(c->L, 3) / std::pow((double)N, 6);
    for (int b = 0; b < nbins; ++b) {
        const double cnt = out[2 * nbins + b];
        n_modes[b] = (int64_t)cnt;
        k_mean[b] = cnt > 0 ? kf * out[nbins + b] / cnt : std::nan("");
        pk[b] = cnt > 0 ? norm * out[b] / cnt : std::nan("");
    }
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
    out->ms_tcola = 0.0;
    if (c->tc_timed && cudaEventQuery(c->tc_ev[1]) != cudaErrorNotReady) {
        float t = 0;
        if (cudaEventSynchronize(c->tc_ev[1]) == cudaSuccess &&
            cudaEventElapsedTime(&t, c->tc_ev[0], c->tc_ev[1]) == cudaSuccess)
            out->ms_tcola = t;
        cudaGetLastError();
    }
    return SCOLA_OK;
}

}  // extern "C"
