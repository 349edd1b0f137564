// Internal declarations shared by the translation units of libscola.
// Device data layout (all FP32 unless noted; boxes concatenated in box-id order):
//   particle arena  12 x P   rows s_x s_y s_z | p_x p_y p_z | psi1_x.. | psi2_x..
//                            (SoA rows, P = sum_b Nsc_b^3, box-local order)
//   dep_acc         uint64 fixed-point CIC counts (2^-32 units) of one group of boxes
//                   (sized to stay in L2; reused by every group, zero between uses)
//   work, work2     sum_b Ng_b^3 interior meshes (transform ping-pong; the deposit
//                   writes the Poisson source delta' into work2)
//   phi             sum_b (Ng_b+4)^3 padded potential (interior + 2 ghost layers)
//   shell           sum_b S_b compact Dirichlet shell values, S_b = (Ng+4)^3 - Ng^3
//   dst tables      per distinct Ng: the sine matrix (transposed, padded rows)
//                   and the Dirichlet eigenvalues
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "scola.h"

namespace scola {

constexpr int kChunk = 256;       // particles per CTA in particle kernels
constexpr int kTC = 32;           // transform columns per tile in the DST passes
constexpr int kXS = kTC + 4;      // shared-memory row stride of a column tile
constexpr int kTcTileRows = 256;  // data rows per tensor-core DST tile (the MMA N)
constexpr double kFix = 4294967296.0;  // 2^32: fixed-point scale of CIC weights
constexpr long long kDepositGroupCells = 6 << 20;   // counts per deposit group (48 MB)

struct BoxDesc {
    int Nsc, Ng, Nbuf, tbl;       // tbl: index of the DST table for this Ng
    int tx, ty, tz;
    int nbe;                      // sorted deposit: key bricks per axis, ceil(Ng / 16) + 1
    long long p_off;              // first particle in the arena
    long long m_off;              // first interior mesh cell
    long long pp_off;             // first padded mesh cell
    long long sh_off;             // first compact shell value
    float dq, dg, inv_dg, q2u;    // q2u = dq / dg
    float nbar_inv;               // (Ng / Nsc)^3
    int key_off;                  // sorted deposit: first key of the box (8 nbe^3 keys per box)
    int gpad;                     // ghost layers per side of the padded potential: 2 N_ghost = FDA order
    int fda;                      // FDA order 2, 4, 6
    double dg_d, origin_d[3];     // FP64 box geometry (cell size, origin of the box frame)
    double inv_2ng_d;             // 1 / (2 Ng) in FP64 (the C.3 shell stencil's offsets)
};

struct Chunk {                    // one CTA of a particle- or cell-parallel kernel
    int box;
    int start;
};

struct DstTable {                 // offsets into the device table arena (floats)
    int Ng;
    int LS;                       // padded row length of the transposed sine matrix (32 R)
    long long st_off;             // ST[i * LS + l] = sin(pi (l+1)(i+1) / (Ng+1))
    long long lam_off;            // lambda[l], l = 0..Ng-1
};

struct TcGroup {                  // one tensor-core DST launch group: boxes sharing Ng
    int Ng, Npad, nkc, nstage;
    int nstage_zm;                // stages of the plane-major z inverse (three-pass solve)
    Chunk *tiles;                 // device (box, kTcTileRows-row tile of the box)
    int ntiles;
    Chunk *planes;                // device (box, plane n) items of the plane pass (three-pass solve)
    int nplanes;
    long long s_off;              // FP32 sine matrix Npad x (32 nkc) in table_arena
    long long lam_off;            // eigenvalues in table_arena
};

struct RxGroup {                  // one radix DST launch group: boxes sharing Ng
    int Ng, P, L, logL, R;        // DFT length P = Ng + 1, Bluestein length L, pencil pairs per tile
    Chunk *tiles;                 // device (box, tile of 2 R rows of the box)
    int ntiles;
    long long w_off, bk_off, tw_off, sn_off, lam_off;   // tables in table_arena
};

struct KickDrift {                // FP32 copies of FP64 host coefficients for one force time
    float kF, k1, k2;             // p += kF F + k1 psi1 + k2 psi2
    float alpha, d1, d2;          // s += alpha p + d1 psi1 + d2 psi2
    int drift;                    // 0 on the last force evaluation
};

struct TimeTable {                // FP64 App. B coefficients
    std::vector<double> a, a_half, D1, D2, beta, kick_from, kick_to, alpha, dD1, dD2;
    double D1_i, D2_i, D1_f, D2_f, dD1da_f, dD2da_f, Hconf_f;
};

// ---- host mathematics (host_math.cpp) ----
double conformal_hubble(double a, double Om, double OL);
void growth_factors(double Om, double OL, const std::vector<double> &a, std::vector<double> &D1,
                    std::vector<double> &D2, std::vector<double> &dD1da, std::vector<double> &dD2da);
double alpha_tilde(double ai, double af, double aK, double Om, double OL, double nLPT);
double beta_tilde(double ai, double af, double aD, double Om, double OL, double nLPT);
TimeTable build_time_table(const scola_params &p);
double bbks_transfer(double k, double Om, double h);   // BBKS T(k), Gamma = Om h
double bbks_amplitude(double Om, double h, double ns, double sigma8);

// ---- context ----
struct Ctx {
    scola_params prm;
    std::vector<int32_t> buffers;
    cudaStream_t stream = nullptr;
    int device = 0;
    int Np = 0, Ntiles = 0, nboxes = 0;
    long long N3 = 0;
    double L = 0, dq = 0, r = 0, p = 0, pk_amp = 0;
    TimeTable tt;

    std::vector<BoxDesc> boxes_h;                     // the bound batch's boxes
    std::vector<DstTable> tables_h;
    std::map<int, int> tbl_of;                        // Ng -> index of its DST table
    long long P = 0, M = 0, MP = 0, SH = 0;
    int max_ng = 0, max_R = 0;

    // streamed batches: the context's boxes (tiling ids [box0, box0 + nbox_all)) are evolved
    // in batches of consecutive boxes; the arenas and work lists hold one batch at a time
    int box0 = 0, nbox_all = 0;
    std::vector<int> batch_first;                     // first box of each batch (context index), then nbox_all
    int bound_batch = -1;                             // the batch the kernels see
    std::vector<BoxDesc> all_boxes_h;                 // every box, laid out within its own batch
    BoxDesc *all_boxes = nullptr;
    long long P_all = 0, M_all = 0;                   // particles and interior cells of all boxes

    // device (the bound batch)
    BoxDesc *boxes = nullptr;
    DstTable *tables = nullptr;
    float *table_arena = nullptr;
    Chunk *pchunks = nullptr;  int n_pchunks = 0;     // box particles
    Chunk *tchunks = nullptr;  int n_tchunks = 0;     // tile particles (scatter)
    Chunk *shchunks = nullptr; int n_shchunks = 0;    // shell cells
    Chunk *zitems = nullptr;   int n_zitems = 0;      // z-pencil tiles
    Chunk *citems = nullptr;   int n_citems = 0;      // (plane, column-tile) items
    Chunk *mchunks = nullptr;  int n_mchunks = 0;     // interior mesh cells
    long long sin_half_off = 0, sin_full_off = 0;     // LPT-grid sine tables in table_arena
    long long amp_off = 0;                            // colouring amplitude per integer |n|^2
    long long lap1_off = 0, grad1_off = 0;            // FDA order 4/6: 1D Laplacian and gradient symbols
    // first entry of each box in every work list (size nboxes + 1), for per-tile launches
    std::vector<int> pbeg, shbeg, zbeg, cbeg, mbeg;
    std::vector<int> dep_groups;                      // first box of each deposit group, then nboxes
    int num_sms = 1, dst_ctas_per_sm = 1;
    bool use_tc = false;                              // tensor-core (3xTF32) DST passes
    bool dst_auto = false, dst_tuned = false;         // SCOLA_DST_AUTO: the autotuner picks use_tc
    bool tc_lo_lo = false;                            // four-product TF32 form
    unsigned long long tc_stall_ns = 0;               // > 0 only inside scola_selftest_wait_timeout
    std::vector<TcGroup> tc_groups;
    Chunk *tc_tiles = nullptr;
    std::vector<int> tc_tile_beg, tc_tile_end;        // each box's tile range in tc_tiles
    bool tc3 = false;                                 // the three-pass tensor-core solve
    bool tc3_ok = false;                              // every Ng allows it (plane_supported)
    Chunk *tc_planes = nullptr;                       // plane items of every group
    std::vector<int> tc_plane_beg;                    // each box's first plane item
    bool rx = false;                                  // the radix (Bluestein) DST passes
    bool rx_ok = false;                               // set up (SCOLA_DST_RADIX, or an AUTO candidate)
    std::vector<RxGroup> rx_groups;
    Chunk *rx_tiles = nullptr;
    std::vector<int> rx_tile_beg, rx_tile_end;        // each box's tile range in rx_tiles
    int view_box = -1;                                // >= 0: launches restricted to this box
    int *dev_err = nullptr;                           // set by kernels whose bounded waits expired
    float *part = nullptr;
    unsigned long long *dep_acc = nullptr;
    // sorted deposit (k_deposit_sorted.cu): per-key counts, slice offsets, fill cursors; the
    // entries (one per box particle at most); the real bricks (box, brick in box)
    int deposit_form = 0;                             // 0: sorted bricks, 1: L2 fixed-point atomics
    int deposit_threads = 512;                        // threads per brick CTA of the sorted form
    int deposit_split = 0;                            // sorted form's counters: 64-bit, 32-bit halves
                                                      // with a carry (1), 16-bit halves reduced (2)
    bool tuned = false;                               // the autotuner has picked the forms above
    // per-tile final scale factors: per box of the bound batch and force evaluation k, the
    // FP32 coefficients [kF (forward, x D1), k1, k2, alpha, d1, d2, 1/D1, beta (adjoint kF)] at
    // coef[(box (nsteps + 1) + k) 8], and the L+ factors [c1, c2] at coefL[2 box]; null
    // when every tile ends at a_f (the kernels then take the uniform scalars)
    float *coef = nullptr, *coefL = nullptr;
    int coef_nk = 0;
    int *kcount = nullptr, *koffs = nullptr, *kcursor = nullptr;
    float4 *sentries = nullptr;
    Chunk *sbricks = nullptr;  int n_sbricks = 0;
    std::vector<int> sbbeg;
    float *work = nullptr, *work2 = nullptr, *phi = nullptr, *shell = nullptr;

    // full-box LPT stage
    float *g[4] = {nullptr, nullptr, nullptr, nullptr};
    float *phi1 = nullptr, *phi2 = nullptr, *psi1 = nullptr, *psi2 = nullptr;
    cufftComplex *ck = nullptr, *cp = nullptr, *ct = nullptr;
    cufftHandle plan_r2c = 0, plan_c2r = 0;
    bool have_plans = false;
    unsigned long long *dens_acc = nullptr;

    // periodic full-box tCOLA (scola_tcola; the study-mode records of scola_forward):
    // Ngf = mesh_ratio Np cells per side; particle state 6 x N3 (s, p_res rows, global-id
    // order); fixed-point counts and FP32 work grids of Ngf^3; per force evaluation K the
    // recorded delta_K and Phi_K ((nsteps + 1) x Ngf^3 each, for the study flags set)
    int tc_ng = 0;
    long long tc_n3 = 0, tc_lap_off = 0;              // tc_lap_off: 1D FDA-2 symbol per index in table_arena
    float *tc_part = nullptr, *tc_delta = nullptr, *tc_phi = nullptr;
    unsigned long long *tc_acc = nullptr;
    cufftComplex *tc_dk = nullptr, *tc_dk2 = nullptr;   // half-spectrum work grids (N^2 (N/2 + 1))
    long long tc_fft_tw_off = 0, tc_fft_w_off = 0, tc_fft_bk_off = 0;   // FFT tables in table_arena
    long long fft_w256_off = 0;                       // the radix-16 second-stage twiddles (fft_util.cuh)
    float *rec_delta = nullptr, *rec_phi = nullptr;

    // adjoint (scola_set_checkpointing / scola_backward)
    bool checkpointing = false, have_forward = false;
    // checkpoints: every ckpt_every-th force evaluation k keeps the displacements (ckpt_every
    // = 1: 3 x P floats per slot, every evaluation) or the displacements and momenta
    // (ckpt_every > 1: 6 x P per slot; the reverse sweep replays each segment of ckpt_every
    // evaluations from its slot into seg and restores the final state from fin)
    int ckpt_every = 1;
    float *ckpt = nullptr;
    // with every-evaluation checkpoints, also each evaluation's padded potential (cap_MP floats
    // per slot) where the slots fit half of the free device memory: the reverse sweep restores
    // it instead of recomputing the deposit and the Poisson solve
    float *ckpt_phi = nullptr;
    float *seg = nullptr, *fin = nullptr;
    long long cap_P = 0, cap_M = 0, cap_MP = 0, cap_SH = 0;   // the largest batch's arena sizes
    float *adj = nullptr;                             // 15 x P backward particle state
    float *lamG = nullptr, *lam_phi_pad = nullptr, *adj_in = nullptr, *adj_out = nullptr;
    float *lam_shell = nullptr, *lamPsi1 = nullptr, *lamPsi2 = nullptr;
    float *lam_phi1 = nullptr, *lam_phi2 = nullptr, *d2 = nullptr, *lam_d2 = nullptr;
    Chunk *ppchunks = nullptr; int n_ppchunks = 0;    // padded mesh cells

    cudaGraphExec_t evolve_exec = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool lpt_done = false, setup_done = false;
    scola_stats stats{};
    long long launches = 0;
};

// ---- kernel launchers (k_*.cu); all enqueue on ctx.stream ----
cudaError_t launch_white_noise(Ctx &c, unsigned long long seed, float *w);
cudaError_t launch_colour(Ctx &c, cufftComplex *ck);
cudaError_t launch_inv_laplacian(Ctx &c, const cufftComplex *in, cufftComplex *out, float scale);
cudaError_t launch_second_derivative(Ctx &c, const cufftComplex *in, cufftComplex *out, int i, int j);
cudaError_t launch_source_init(Ctx &c, const float *xx, const float *yy, const float *zz, float *S);
cudaError_t launch_source_sub(Ctx &c, const float *t, float *S);
cudaError_t launch_gradient(Ctx &c, const float *phi, float *psi);

cudaError_t launch_box_init(Ctx &c);
cudaError_t launch_shell(Ctx &c);
// Ghost layers of the padded potential <- D1 x shell.  The solve runs on Phi / D1(a_K), so
// the ghost layers hold the unscaled shell (D1 = 1), written once per forward run.
cudaError_t launch_pad(Ctx &c, float D1);
// counted: the key counts of s were made by the kick-drift that moved the particles (sorted
// form, batched graph); otherwise the deposit counts them itself
// inv_D1: the Poisson source is delta / D1(a_K) minus the boundary term of the unscaled
// shell, so that the solve gives Phi / D1 (delta_out receives delta itself)
// k >= 0: force evaluation k of the evolution (with per-tile final scale factors the
// kernels take each box's 1/D1 from the coefficient table); k < 0: inv_D1 for every box
cudaError_t launch_deposit(Ctx &c, const float *s, long long stride, float inv_D1, float *delta_out = nullptr,
                           bool counted = false, int k = -1);
cudaError_t launch_deposit_atomic(Ctx &c, const float *s, long long stride, float inv_D1, float *delta_out, int k);
cudaError_t launch_deposit_sorted(Ctx &c, const float *s, long long stride, float inv_D1, float *delta_out,
                                  bool counted, int k);
cudaError_t clear_key_counts(Ctx &c);
cudaError_t init_pm_kernels(Ctx &c);
cudaError_t init_deposit_kernels();
int tc_plan_stages(int Ng, int &Npad, int &nkc, bool zm = false);
bool plane_supported(int Ng);    // the three-pass solve: Ng <= 96, Ng % 4 == 0
cudaError_t init_plane_kernel();
cudaError_t launch_plane_pass(Ctx &c, const std::vector<TcGroup> &groups, const float *in, float *out);
// radix DST (k_dst_radix.cu): plan of one Ng, its host tables appended to the arena
void rx_plan(int Ng, int &P, int &L, int &logL, int &R);
bool rx_supported(int Ng);
void rx_tables(RxGroup &G, std::vector<float> &arena);
cudaError_t init_rx_kernels();
cudaError_t launch_poisson_rx_pass(Ctx &c, int pass);
cudaError_t launch_poisson_rx_buffers(Ctx &c, const float *in, float *w1, float *w2, float *out_pad);
bool tc_supported(int Ng);
bool tc_folded(int Ng);          // Ng > 128: the mirror-symmetric half-size form
bool tc_ragged(int Ng);          // rows not 16-byte pitched for TMA: plain loads and stores
cudaError_t init_tc_kernels();
cudaError_t launch_poisson_tc(Ctx &c);
cudaError_t launch_poisson_tc_pass(Ctx &c, int pass);
cudaError_t launch_poisson_tc_buffers(Ctx &c, const float *in, float *w1, float *w2,
                                      float *out_pad);
cudaError_t launch_poisson_buffers(Ctx &c, const float *in, float *w1, float *w2,
                                   float *out_pad);
cudaError_t launch_poisson(Ctx &c);
cudaError_t launch_poisson_pass(Ctx &c, int pass);
// F = D1 x gradient of the stored potential Phi / D1
cudaError_t launch_interp(Ctx &c, const float *s, long long stride, float *F, float D1);
cudaError_t launch_scaled_copy(Ctx &c, const float *in, float *out, long long n, float a);
// count_keys: also count the sorted deposit's keys of the drifted particles (into cleared
// counts) for the next force evaluation
cudaError_t launch_kick_drift(Ctx &c, const KickDrift &kd, bool count_keys = false, int k = -1);
cudaError_t launch_scatter(Ctx &c, float *x, float *p);
cudaError_t launch_box_ids(Ctx &c, int64_t *gid);
// per box of the bound batch: inside CIC weight (2^-32 fixed point) and clamped-particle count
cudaError_t launch_box_mass(Ctx &c, const float *s, unsigned long long *mass, int *escaped);
cudaError_t launch_final_density(Ctx &c, const float *x, float *delta);
// Binned |delta_k|^2 sums of a half spectrum: out = [psum, sqrt(n^2) sum, count] x nbins;
// scratch holds 3 x rows x nbins doubles; rows = CTAs of the partial pass.
cudaError_t launch_spectrum(Ctx &c, const cufftComplex *dk, const int *bin_of_n2, int nbins, double *scratch,
                            int rows, double *out);
constexpr int kMaxSpectrumBins = 2048;

// periodic tCOLA (k_tcola.cu): particle init, deposit into the counts, density (clears the
// counts), kick-drift reading the potential phi, final x and p
cudaError_t launch_tc_init(Ctx &c);
cudaError_t launch_tc_deposit(Ctx &c);
cudaError_t launch_tc_density(Ctx &c, float *delta);
// the periodic Poisson solve delta -> Phi on the tCOLA grid (k_tcola_fft.cu, five passes)
void tc_fft_plan(int N, int &L, int &logL, int &R, bool &blue);
bool tc_fft_supported(int N);
void tc_fft_tables(int N, std::vector<float> &arena, long long &tw_off, long long &w_off, long long &bk_off);
cudaError_t init_tc_fft_kernels();
cudaError_t launch_tc_poisson(Ctx &c, const float *delta, float *phi);
cudaError_t launch_tc_kick_drift(Ctx &c, const float *phi, const KickDrift &kd);
cudaError_t launch_tc_final(Ctx &c, float *x, float *p);
// study inputs of the bound batch's boxes: the Poisson source from a full-grid delta
// (into work2), the ghost layers from a full-grid Phi (into the padded potential)
cudaError_t launch_true_source(Ctx &c, const float *delta, float inv_D1);
cudaError_t launch_true_pad(Ctx &c, const float *phi, float inv_D1);

cudaError_t launch_adj_colour(Ctx &c, const cufftComplex *in, cufftComplex *out);
cudaError_t launch_adj_final(Ctx &c, const float *lam_delta, float *adj);
// tile particles' initial adjoint state from the cotangents of the global x and p (either null)
cudaError_t launch_adj_final_xp(Ctx &c, const float *lam_x, const float *lam_p, float *adj);
// the periodic CIC adjoint of the final density over the global positions
cudaError_t launch_density_vjp(Ctx &c, const float *x, const float *lam_delta, float *lam_x);
// k >= 0 with per-tile final scale factors: each box's factors of evaluation k (coef table)
cudaError_t launch_adj_kick_drift(Ctx &c, float *adj, const KickDrift &kd, int k = -1);
cudaError_t launch_adj_interp(Ctx &c, const float *s, float *adj, float *lamG, float D1, int k = -1);
cudaError_t launch_adj_div(Ctx &c, const float *lamG, float *lam_phi_pad, float *interior_out);
cudaError_t launch_adj_shell(Ctx &c, const float *lam_phi_pad, const float *lam_src_pad, float D1,
                             float *lam_shell, int k = -1);
cudaError_t launch_adj_deposit(Ctx &c, const float *s, const float *lam_src_pad, float *adj);
cudaError_t launch_adj_init_scatter(Ctx &c, const float *adj, float *lamPsi1, float *lamPsi2);
cudaError_t launch_adj_shell_to_phi1(Ctx &c, const float *lam_shell, float *lam_phi1);
cudaError_t launch_neg_div(Ctx &c, const float *g, int accumulate, float *out);
cudaError_t launch_adj_source(Ctx &c, const float *lamS, const float *d2, float *lam_d2);
cudaError_t launch_spec_d2_accumulate(Ctx &c, const cufftComplex *in, cufftComplex *acc, int i, int j);

void set_error(const std::string &msg);
// Records "<step>: <CUDA error string>" as the context's error detail and returns e; the
// caller's own report then keeps this detail (see CK in capi.cu).
cudaError_t step_error(const char *step, cudaError_t e);

}  // namespace scola
