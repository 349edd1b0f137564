/*
 * scola.h - C ABI of the GB300 (sm_103a) library for the perfectly parallel
 * spatial-COLA (sCOLA) method of Leclercq et al., arXiv:2003.04925.
 *
 * What the library computes (the paper's statement of the problem, Sec. 3):
 * a periodic box of side L holds Np^3 particles on a Lagrangian lattice.
 * From a white-noise field the library builds the initial density
 * (Sec. 3.1, A.1) and the 2LPT potentials and displacements (Sec. 2.1,
 * Eqs. 2-6, A.2), splits the lattice into Ntiles^3 tiles with a buffer of
 * Nbuf particles around each (Sec. 3.2, B.1), evolves every sCOLA box
 * independently with a particle-mesh COLA integrator whose Poisson solve uses
 * Dirichlet boundary values from the linearly evolving potential (Sec. 3.3,
 * 3.4, Eq. 23, App. A-C), and writes the tile particles back to global
 * arrays (B.2).  Every step of this path runs in the library's own CUDA
 * kernels except the full-box Fourier transforms of the initial-condition
 * stage and of its adjoint, which call cuFFT once per run (the paper's code
 * calls FFTW there, Sec. 3.1).
 *
 * Conventions used by every entry point:
 *   - units: Mpc/h, time in 1/H0 with H0 = 1, time variable the scale factor a;
 *   - particle (i, j, k), k fastest, has id (i*Np + j)*Np + k and Lagrangian
 *     position q = ((i + 1/2), (j + 1/2), (k + 1/2)) * L/Np;
 *   - tile (tx, ty, tz) has box id (tx*Ntiles + ty)*Ntiles + tz;
 *   - grids are C-ordered [i][j][k] FP32 arrays, k fastest;
 *   - "device" pointers are CUDA device (or managed) memory owned by the
 *     caller and must stay valid until the stream work completes;
 *   - every call that launches work enqueues it on the context's stream and
 *     returns without synchronising, unless its comment says otherwise;
 *   - no call throws; each returns a scola_status.  On SCOLA_ERR_CUDA the
 *     CUDA error string is available from scola_last_error().
 *
 * Thread safety: a context may be used by one host thread at a time.
 */
#ifndef SCOLA_H
#define SCOLA_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum scola_status {
    SCOLA_OK = 0,
    SCOLA_ERR_INVALID_ARG = 1,   /* a parameter violates the problem statement */
    SCOLA_ERR_UNSUPPORTED = 2,   /* valid in the paper, not built here (e.g. FDA order 4/6) */
    SCOLA_ERR_OOM = 3,           /* a device allocation failed */
    SCOLA_ERR_CUDA = 4,          /* a CUDA or cuFFT call failed; see scola_last_error() */
    SCOLA_ERR_STATE = 5,         /* call made in the wrong order (e.g. force before setup) */
    SCOLA_ERR_TIMEOUT = 6        /* a kernel's bounded wait expired (see scola_device_status) */
} scola_status;

typedef enum scola_dst_variant {
    SCOLA_DST_SIMT = 0,          /* dense sine-matrix pencils on FP32 CUDA cores */
    SCOLA_DST_TC_3XTF32 = 1,     /* the same products on tcgen05 tensor cores, 3xTF32 split;
                                    every 2 <= Ng <= 240 (the sine matrix resident in shared
                                    memory, folded by its mirror symmetry for Ng > 128) */
    SCOLA_DST_TC_4XTF32 = 3,     /* as 1, plus the lo x lo product (four TF32 products) */
    SCOLA_DST_TC_3PASS = 4,      /* the products in three mesh passes instead of six: z forward
                                    (3xTF32); every z-frequency plane transformed along y and x,
                                    divided and transformed back in shared memory (3xFP16, each
                                    pencil scaled by a power of two into FP16's range: the same
                                    ~22 bits as 3xTF32 at twice its rate); z inverse (3xTF32).
                                    Every Ng <= 96 with Ng % 4 == 0 (UNSUPPORTED otherwise) */
    SCOLA_DST_RADIX = 5,         /* fast sine transforms on FP32 CUDA cores, O(Ng log Ng) per
                                    pencil: each DST-I of length Ng from a real DFT of length
                                    Ng + 1 (two pencils per complex transform), done by
                                    Bluestein's chirp convolution with radix-16 FFTs of a power-of-two
                                    length in shared memory; every 1 <= Ng <= 256 */
    SCOLA_DST_AUTO = 2           /* the fastest of the tensor-core forms (six passes, and three
                                    where every Ng allows it), the dense FP32 form and the radix
                                    form, timed once on the context's boxes before the first
                                    evolution (where Ng > 222 excludes the dense FP32 form: the
                                    six-pass tensor-core form alone; where Ng > 240 excludes the
                                    tensor cores: the radix form) */
} scola_dst_variant;

typedef enum scola_deposit_form {
    SCOLA_DEPOSIT_AUTO = 0,      /* the faster of the forms below on this context's boxes, timed
                                    once with CUDA events before the first evolution */
    SCOLA_DEPOSIT_SORTED = 1,    /* particles sorted by 16^3-cell brick, each brick's counts
                                    reduced in shared memory (256 or 512 threads, 64-bit
                                    counters or 32-bit halves: timed) */
    SCOLA_DEPOSIT_ATOMIC = 2     /* 64-bit fixed-point atomics into an L2-resident scratch,
                                    boxes taken in groups whose counts fit L2 */
} scola_deposit_form;

typedef enum scola_time_stepping {
    SCOLA_STEPPING_MODIFIED = 0, /* modified KDK factors with u(a) = a^nLPT (App. B; the paper's runs) */
    SCOLA_STEPPING_STANDARD = 1  /* standard KDK factors: interval integrals of the drift and
                                    kick prefactors (App. B) */
} scola_time_stepping;

typedef enum scola_study_mode {   /* bit flags (Sec. 4.3 approximation tests) */
    SCOLA_STUDY_NONE = 0,            /* the method: delta_int = delta^sCOLA, Phi_BCs = Phi_LEP */
    SCOLA_STUDY_TRUE_DENSITY = 1,    /* delta_int = delta of the periodic tCOLA run */
    SCOLA_STUDY_TRUE_POTENTIAL = 2   /* Phi_BCs = Phi of the periodic tCOLA run */
} scola_study_mode;

typedef enum scola_batch_mode {
    SCOLA_BATCH_ALL = 0,         /* every box in each launch (batched form) */
    SCOLA_BATCH_PER_TILE = 1     /* one box per launch, boxes in turn (plain per-tile form) */
} scola_batch_mode;

/*
 * Problem statement.  Field names follow the paper's nomenclature (Sec. 3,
 * nomenclature table):
 *   L            full box side [Mpc/h]
 *   Np           particles per side; the LPT grid has N = Np cells per side
 *   Ntiles       tiles per side; Np must be a multiple of Ntiles (Sec. 3.2)
 *   Nbuf         buffer particles per side, the same for every tile
 *   buffers      optional per-tile buffer widths (host array of Ntiles^3,
 *                box-id order), copied by scola_create; NULL = use Nbuf
 *   mesh_ratio   PM cells per particle spacing: Ng = mesh_ratio * Np,sCOLA
 *   Ng           explicit PM grid size per side (uniform buffers only);
 *                0 = use mesh_ratio.  Ng >= Np,sCOLA (Sec. 3.3, C.3)
 *   Om, OL       matter and Lambda density parameters (Ok = 1 - Om - OL)
 *   h, ns, sigma8  BBKS power spectrum P = A k^ns T^2(k / (Om h)), normalised
 *                to sigma8 at a = 1
 *   a_i, a_f     initial (2LPT) and final scale factors
 *   nsteps       COLA drift steps, linear in a (nsteps + 1 force evaluations)
 *   nLPT         exponent of the modified time stepping u(a) = a^nLPT
 *                (App. B, Eq. 60); the paper uses -2.5
 *   fda_order    finite-difference order 2, 4 or 6 of every gradient and Laplacian
 *                (Sec. 3.1; N_ghost = fda_order / 2): the padded potential has fda_order
 *                ghost layers per side, the boundary source of Eq. 62 reaches N_ghost
 *                cells inside, and the DST solve uses App. C's order-n eigenvalues.
 *                The adjoint is built for order 2
 *   dst_variant  one of scola_dst_variant
 *   batch_mode   one of scola_batch_mode (same results, different launch shapes)
 *   deposit_form one of scola_deposit_form.  Every form sums the CIC weights as
 *                2^-32 fixed-point integers, so all give the same density bit for
 *                bit; the choice changes only the speed
 *   batch_boxes  the context's boxes are evolved in batches of consecutive boxes that
 *                share one set of per-box arenas (boxes never communicate, so any
 *                batching gives the same result bit for bit).  0 = as many boxes as
 *                fit in the device memory left after the full-box LPT stage and a
 *                reserve of 2 x 28 bytes per particle (the caller's w, x, p and the
 *                host-copy buffers of scola_forward_host) plus 1 GiB; the batch count
 *                is then raised to a divisor of the box count where batches stay at
 *                least half full.  A context with more than one batch runs
 *                scola_forward, scola_forward_host, scola_final_density, the adjoint
 *                calls and the host-only calls; the per-stage and inspection calls need
 *                one batch (they return UNSUPPORTED otherwise)
 *   time_stepping one of scola_time_stepping
 *   a_final      optional per-tile final scale factors (host array of Ntiles^3, box-id
 *                order, each > a_i), copied by scola_create; NULL = a_f for every tile.
 *                Boxes never communicate, so each tile may stop at its own scale factor
 *                (light-cone scheduling, Sec. 5): tile t takes nsteps steps linear in a
 *                from a_i to a_final[t], and its particles leave scola_forward at that
 *                time (positions and momenta with L+ at a_final[t]).  All boxes still go
 *                through each launch together
 *   study_mode   bit flags of scola_study_mode (Sec. 4.3).  0 runs the method.  Otherwise
 *                scola_forward first runs the periodic full-box tCOLA of scola_tcola and
 *                keeps its density and potential at every force evaluation, then evolves
 *                the boxes with the interior density (TRUE_DENSITY) and/or the ghost-layer
 *                potential (TRUE_POTENTIAL) taken from those fields instead of the box
 *                deposit and the LEP shell.  The box meshes must coincide with cells of the
 *                full-box mesh (Ng = mesh_ratio * Np,sCOLA), FDA order 2, no a_final, no
 *                adjoint (UNSUPPORTED otherwise).  The records take 4 (nsteps + 1)
 *                (mesh_ratio Np)^3 bytes per flag.  With both flags the boxes reproduce the
 *                tCOLA run up to rounding.  Only scola_forward(_host) is affected
 *   lpt_order    2: initial conditions and the COLA frame from 2LPT (Eqs. 5-6, 39);
 *                1: the Zel'dovich approximation (Psi2 = 0: first-order displacements,
 *                frame and L+/L- from Psi1 alone, Sec. 2.2)
 *   box_first, box_count  evolve only boxes [box_first, box_first + box_count)
 *                of the tiling (both 0: all boxes).  Boxes never communicate
 *                (Sec. 3.2), so several contexts (for example one per GPU) can
 *                split a run; each writes only its own tiles' particles and
 *                leaves the other entries of x and p untouched.
 */
typedef struct scola_params {
    double L;
    int32_t Np;
    int32_t Ntiles;
    int32_t Nbuf;
    int32_t mesh_ratio;
    int32_t Ng;
    int32_t fda_order;
    int32_t dst_variant;
    int32_t nsteps;
    int32_t batch_mode;
    int32_t box_first;
    int32_t box_count;
    int32_t deposit_form;        /* one of scola_deposit_form */
    int32_t batch_boxes;         /* boxes per streamed batch; 0 = as many as fit */
    int32_t time_stepping;       /* one of scola_time_stepping */
    int32_t lpt_order;           /* 2: 2LPT frame (the paper's runs); 1: Zel'dovich frame */
    int32_t study_mode;          /* scola_study_mode flags; 0 = the method */
    double Om, OL, h, ns, sigma8;
    double a_i, a_f;
    double nLPT;
    const int32_t *buffers;
    const double *a_final;       /* per-tile final scale factors (light-cone scheduling) or NULL */
} scola_params;

typedef struct scola_ctx scola_ctx;

/* Run statistics of the last scola_forward (or scola_pm_force) call. */
typedef struct scola_stats {
    int32_t nboxes;
    int64_t box_particles;        /* sum over boxes of Np,sCOLA^3 */
    int64_t mesh_cells;           /* sum over boxes of Ng^3 */
    int32_t force_evaluations;    /* nsteps + 1 */
    double r, p;                  /* over-simulation r (Eq. 20), parallelisation potential p (Eq. 21) */
    double ms_lpt;                /* initial-condition and 2LPT stage, device time (on the
                                     first call, plus the deposit autotuner's runs) */
    double ms_evolve;             /* gather + evolution + scatter, device time */
    int64_t kernel_launches;      /* kernels launched by the last forward call */
    int32_t deposit_form;         /* the form in use: SCOLA_DEPOSIT_SORTED or _ATOMIC (0 before
                                     the first scola_forward / scola_setup_boxes) */
    int32_t deposit_threads;      /* threads per brick CTA of the sorted form, else 0 */
    int32_t deposit_split;        /* the sorted form's counters: 0 64-bit, 1 32-bit halves with a
                                     carry, 2 16-bit halves with reductions (exact while a brick
                                     holds at most 65535 entries; busier bricks use 1) */
    double ms_deposit_candidates[5]; /* autotuner timings of one deposit (all boxes of the first
                                     batch, or its box 0 in the per-tile form): sorted/256,
                                     sorted/512, sorted/256 with 32-bit halves, atomic;
                                     0 = not timed */
    int32_t batches;              /* streamed batches per forward run */
    int32_t batch_boxes;          /* boxes per batch (the last may hold fewer) */
    double ms_tcola;              /* periodic tCOLA run (scola_tcola, or the study-mode records
                                     of scola_forward), device time; 0 if none ran */
    int32_t dst_form;             /* the Poisson-solve form in use (scola_dst_variant) once chosen:
                                     the requested one, or the autotuner's pick under AUTO
                                     (0 until the first scola_forward / scola_setup_boxes) */
    double ms_dst_candidates[4];  /* AUTO: autotuner timings of one Poisson solve: tensor cores
                                     in six passes, dense FP32, tensor cores in three passes,
                                     radix FP32; 0 = not timed */
    int32_t adjoint_potentials_kept; /* 1: with checkpoints at every force evaluation the
                                     forward run also keeps each evaluation's padded potential
                                     (they fit half of the free device memory), and the
                                     backward pass restores it instead of recomputing the
                                     deposit and the Poisson solve */
} scola_stats;

/*
 * Validate the problem, compute the FP64 cosmology (growth factors, COLA
 * time coefficients, power-spectrum amplitude) on the host, and allocate the
 * context's device arenas on the current device.
 *   params  problem statement (copied)
 *   stream  cudaStream_t on which all later work is enqueued (NULL = legacy default)
 *   out     receives the new context
 * Errors: INVALID_ARG (Np % Ntiles != 0, Ng < Np,sCOLA, non-positive sizes,
 * a_i >= a_f, nsteps < 1, Np,sCOLA > Np, study_mode outside 0..3), UNSUPPORTED (fda_order
 * not 2, 4 or 6; a study mode with unaligned box meshes, FDA order 4/6 or a_final), OOM, CUDA.
 * Synchronous.
 */
scola_status scola_create(const scola_params *params, void *stream, scola_ctx **out);

/* Free the context and its device arenas.  Synchronises the stream first. */
void scola_destroy(scola_ctx *ctx);

/*
 * The full forward run (Sec. 3, Fig. 1): A.1-A.2 on the full box, B.1 tiling,
 * C.1-C.3 per box, D evolution of every box, B.2 untiling.
 *   w_dev  device, Np^3 FP32 white noise (unit variance per LPT cell)
 *   x_dev  device, Np^3 x 3 FP32, receives final positions in [0, L), id order
 *   p_dev  device, Np^3 x 3 FP32, receives final momenta p = dx/da / calD
 *          (App. A, Eq. 37) including the LPT part (L+, Eq. 55)
 * The evolution is replayed from a CUDA graph captured on the first call.
 */
scola_status scola_forward(scola_ctx *ctx, const float *w_dev, float *x_dev, float *p_dev);

/*
 * Same as scola_forward with HOST buffers: copies w to the device, runs,
 * copies x and p back, and synchronises the stream before returning.
 *   w_host  host, Np^3 FP32; x_host, p_host  host, Np^3 x 3 FP32
 */
scola_status scola_forward_host(scola_ctx *ctx, const float *w_host, float *x_host, float *p_host);

/*
 * The initial-condition and 2LPT stage alone (Sec. 3.1, A.1-A.2; Eqs. 5-6;
 * Psi = FDA-2 gradient at the lattice nodes, App. A below Eq. 39).  Also
 * leaves the fields in the context for scola_setup_boxes.
 *   w_dev     device, Np^3 FP32 white noise
 *   delta_dev, phi1_dev, phi2_dev   device, Np^3 FP32 each, or NULL
 *   psi1_dev, psi2_dev              device, 3 x Np^3 FP32 each ([component][id]), or NULL
 */
scola_status scola_lpt_fields(scola_ctx *ctx, const float *w_dev, float *delta_dev,
                              float *phi1_dev, float *phi2_dev,
                              float *psi1_dev, float *psi2_dev);

/*
 * C.1-C.3 for every box from the fields of the last scola_lpt_fields call:
 * gather Psi1, Psi2 of the box particles, set s = -D1(a_i) Psi1 + D2(a_i) Psi2,
 * p_res = 0 (L-, Eq. 55), and precompute the Dirichlet shell (phi1 trilinearly
 * interpolated to the padded PM cells outside the interior; C.3, Eq. 23).
 * Errors: STATE if scola_lpt_fields has not run.
 */
scola_status scola_setup_boxes(scola_ctx *ctx);

/*
 * One PM force evaluation in every box (Sec. 3.4): B^sCOLA deposit of the
 * given displacements, Dirichlet DST-I Poisson solve with
 * Phi_BCs = D1 * shell (Eq. 23, App. C), FDA-2 gradient and CIC
 * interpolation.  Uses the shells of scola_setup_boxes.
 *   s_dev     device, 3 x P FP32 box-particle displacements s = x - q,
 *             [component][box particle], boxes concatenated in box-id order,
 *             box-local particle order (bi*Nsc + bj)*Nsc + bk
 *   D1        growth factor scaling the boundary shell
 *   F_dev     device, 3 x P FP32, receives grad Phi at the particles
 *   delta_dev device, scola_mesh_cell_count() FP32: box b's interior densities
 *             (delta, before the boundary correction) as Ng^3 cells [i][j][k]
 *             from offset m_off[b] of scola_box_offsets, or NULL
 *   phi_dev   device, scola_padded_cell_count() FP32: box b's padded potential
 *             as (Ng+4)^3 cells from offset pp_off[b], or NULL
 * P = scola_box_particle_count().  Errors: STATE before scola_setup_boxes.
 */
scola_status scola_pm_force(scola_ctx *ctx, const float *s_dev, double D1, float *F_dev,
                            float *delta_dev, float *phi_dev);

/* Number of box particles P (sum over the boxes of Np,sCOLA^3) of the bound batch: all
 * boxes of a one-batch context. */
int64_t scola_box_particle_count(const scola_ctx *ctx);

/* Sizes of the interior and padded mesh arrays of the bound batch: the boxes' Ng^3 and
 * (Ng+4)^3 cells at the offsets of scola_box_offsets, with alignment gaps between boxes. */
int64_t scola_mesh_cell_count(const scola_ctx *ctx);
int64_t scola_padded_cell_count(const scola_ctx *ctx);

/*
 * Where each box of the context sits in the mesh arrays (the layout of
 * scola_pm_force's delta and phi outputs).
 *   m_off, pp_off  host, nboxes int64 each: first interior / padded cell of box b
 *   nboxes         the context's box count (scola_get_stats().nboxes)
 * Errors: INVALID_ARG (NULL, nboxes different from the context's).
 */
scola_status scola_box_offsets(const scola_ctx *ctx, int64_t *m_off, int64_t *pp_off, int32_t nboxes);

/*
 * Tile assignment (Sec. 3.2): global particle id of every box particle, in
 * the layout of scola_pm_force (device kernel, bit-exact integer arithmetic).
 *   gid_dev  device, P int64
 */
scola_status scola_box_particle_ids(scola_ctx *ctx, int64_t *gid_dev);

/*
 * Multi-GPU sharding plan (host only, no context needed).  The boxes never communicate
 * (Sec. 3.2), so a run splits into contiguous box ranges, one per GPU, each evolved by its
 * own context (params.box_first / box_count) with no collective on the data path.  The
 * ranges balance the cost Np,sCOLA^3 + Ng^3 of each box: rank r ends its range where the
 * running cost comes within half a box of (r + 1) / world of the total, leaving at least
 * one box for every later rank; the last rank takes the rest.
 *   world        number of ranks, 1 .. Ntiles^3
 *   first, count host, world int32: each rank's range (together every box exactly once)
 * Errors: as scola_create's validation; INVALID_ARG (NULL, world out of range).
 */
scola_status scola_shard_ranges(const scola_params *params, int32_t world, int32_t *first, int32_t *count);

/*
 * Host-side tiling arithmetic (Sec. 3.2, Eqs. 20-21), no context needed.
 *   box_nsc  host, Ntiles^3 int32 or NULL: Np,sCOLA per box
 *   box_ng   host, Ntiles^3 int32 or NULL: Ng per box
 *   r, p     host or NULL: over-simulation and parallelisation potential
 */
scola_status scola_tiling_info(const scola_params *params, int32_t *box_nsc, int32_t *box_ng,
                               double *r, double *p);

/*
 * Final density (Sec. 4.1): periodic CIC of all Np^3 particles on the N^3 LPT
 * grid, delta = rho / nbar - 1.  Deterministic (fixed-point accumulation).
 *   x_dev      device, Np^3 x 3 FP32 positions
 *   delta_dev  device, Np^3 FP32
 */
scola_status scola_final_density(scola_ctx *ctx, const float *x_dev, float *delta_dev);

/*
 * FP64 time-stepping table the kernels use (App. B, Eqs. 52-60), computed on
 * the host without a context or a GPU: growth factors by an adaptive
 * Dormand-Prince integration of the growth equations (Eqs. 44-45), alpha~ by
 * Gauss-Legendre quadrature, beta~ in closed form.
 * For force evaluation k = 0..nsteps (host arrays of nsteps + 1, any may be NULL):
 *   a_force, D1, D2, beta (coefficient of the kick that uses that force);
 * for drift k = 0..nsteps-1 (host arrays of nsteps): alpha, dD1, dD2.
 * Errors: as scola_create's validation.
 */
scola_status scola_time_table(const scola_params *params, double *a_force, double *D1, double *D2,
                              double *beta, double *alpha, double *dD1, double *dD2);

/*
 * Profiling mode: when enabled, the evolution graph is re-captured with an
 * external CUDA event recorded between consecutive kernels of every force
 * evaluation, so that scola_kernel_times can report device time per kernel.
 * Synchronises the stream.  Costs a few microseconds per force evaluation.
 */
scola_status scola_set_profiling(scola_ctx *ctx, int32_t enable);

/*
 * Average device time per launch [ms] of each kernel class in the last
 * forward run made in profiling mode (synchronises on it).  ms_per_launch
 * (host, n >= 8 doubles) receives, in order: deposit (with the boundary source
 * and the clearing of its counters), the Poisson passes 1..6, interpolate +
 * kick + drift.  FP32 form: pass 1 z forward, 2 y forward,
 * 3 x forward + sine-space division + x inverse, 4 y inverse, 5 z inverse,
 * 6 empty.  Tensor-core form: 1 z forward, 2 y forward, 3 x forward +
 * division, 4 z inverse, 5 y inverse, 6 x inverse.
 * Errors: STATE when profiling is off.
 */
scola_status scola_kernel_times(const scola_ctx *ctx, double *ms_per_launch, int32_t n);

/*
 * Average device time per force evaluation [ms] of the stages of the last periodic tCOLA
 * run (scola_tcola, or the study-mode records of scola_forward) made in profiling mode.
 * ms_per_launch (host, n >= 4 doubles) receives: periodic CIC deposit, density (counts ->
 * delta, clearing the counts), Poisson solve (five passes of shared-memory FFTs with the
 * Green's function in the z pass), interpolate + kick + drift.  Errors: STATE when no tCOLA run was profiled.
 */
scola_status scola_tcola_kernel_times(const scola_ctx *ctx, double *ms_per_launch, int32_t n);

/*
 * Synchronises the stream and reports whether a kernel gave up on a bounded
 * wait since the context was created or since the last call that reported one:
 * SCOLA_OK, or SCOLA_ERR_TIMEOUT (results of the affected launch are invalid;
 * the context stays usable), or SCOLA_ERR_CUDA when the sorted deposit's fill
 * pass found more particles for a key than its count pass (nothing is written
 * past the slot range; the densities of that launch are invalid).  A reported
 * condition is cleared.
 */
scola_status scola_device_status(scola_ctx *ctx);

/*
 * Failure-detection self-test (the paper has no counterpart).  Runs one tensor-core DST
 * pass over the context's scratch meshes in which the thread that issues the tensor-core
 * instructions first waits, for wait_seconds, on a barrier that nothing arrives on.  The
 * wait expires, the CTA raises the device error flag, its other roles leave their loops at
 * their next bounded wait, the tensor copies already issued drain (those waits keep their
 * normal 2 s limit), tensor memory is freed and the kernel returns: nothing faults or hangs.
 * Synchronous.  Returns SCOLA_ERR_TIMEOUT when the wait expired as designed (the flag is
 * then cleared, see scola_device_status); the context stays usable and its next forward
 * run is unaffected (the pass wrote only scratch meshes).
 *   wait_seconds  0 < wait_seconds <= 2
 * Errors: INVALID_ARG, UNSUPPORTED (no tensor-core DST, or more than one batch), STATE (no
 * forward run or box set-up yet), CUDA.
 */
scola_status scola_selftest_wait_timeout(scola_ctx *ctx, double wait_seconds);

/* 1 when the context's Poisson solve runs on the tensor cores, else 0 (under
 * SCOLA_DST_AUTO: the autotuner's pick once the first scola_forward or
 * scola_setup_boxes has run; before that, whether the tensor-core form is set up). */
int32_t scola_uses_tensor_cores(const scola_ctx *ctx);

/*
 * Adjoint support.  With checkpointing enabled, scola_forward also stores checkpoints of
 * every box particle's state (see scola_set_checkpoint_interval) and the context keeps the
 * adjoint work arrays.  Batched form, no study mode (UNSUPPORTED otherwise); FDA order 2, 4
 * or 6, 2LPT or Zel'dovich frame, modified or standard KDK factors, common or per-tile final
 * scale factors, one or several streamed batches, any Poisson-solve form.  Synchronises the
 * stream.
 */
scola_status scola_set_checkpointing(scola_ctx *ctx, int32_t enable);

/*
 * How often the forward run checkpoints the particle state for the adjoint (the paper has no
 * counterpart; it keeps long differentiated runs within device memory).  With n force
 * evaluations (nsteps + 1) and P box particles per batch:
 *   every = 1   every evaluation keeps the displacements: 3 n P floats, no recomputation;
 *   every = m   every m-th evaluation keeps displacements and momenta, 6 ceil(n / m) P floats,
 *               plus 3 m P for one replayed segment and 6 P for the final state: the reverse
 *               sweep replays each segment of m evaluations forward from its checkpoint (the
 *               same deterministic kernels, so the same trajectory and the same gradient) at
 *               the cost of one more forward pass;
 *   every = 0   the m that needs the fewest floats (about sqrt(2 n)).
 * With several streamed batches the backward pass replays each batch's evolution from C.1
 * to rebuild its checkpoints (one more forward pass).  The default is 1.  Changing the
 * interval drops any stored checkpoints (the next backward needs a new forward run).
 * Synchronises the stream.  Errors: INVALID_ARG (NULL, every < 0), OOM, CUDA.
 */
scola_status scola_set_checkpoint_interval(scola_ctx *ctx, int32_t every);

/* The checkpoint interval in use (1 by default). */
int32_t scola_checkpoint_interval(const scola_ctx *ctx);

/*
 * Vector-Jacobian product of the whole forward run: the gradient, with respect to the white
 * noise, of a loss of the final particle positions and momenta of the last scola_forward run
 * on this context (made with checkpointing on).  The outputs of that run are x = (q + s) mod L
 * (Sec. 2.1, Eq. 1, B.2) and p = p_res + a_f^2 calH(a_f)(-dD1/da Psi1 + dD2/da Psi2) (L+,
 * Eq. 55) of every particle, so the sweep starts from lam_s = dL/dx, lam_p_res = dL/dp and the
 * L+ transpose on each tile particle (buffer particles leave no output).
 *   lam_x_dev  device, Np^3 x 3 FP32: dLoss/dx in the layout of scola_forward's x, or NULL (zero)
 *   lam_p_dev  device, Np^3 x 3 FP32: dLoss/dp in the layout of scola_forward's p, or NULL (zero)
 *   lam_w_dev  device, Np^3 FP32, receives dLoss/dw
 * Hand-written vector-Jacobian products of every step, in reverse: the untiling and L+, the
 * KDK sequence with the recomputed mesh force at each checkpoint (interpolation weights,
 * gradient mesh, the self-adjoint Dirichlet solve, the boundary source and ghost layers,
 * deposit weights, App. B-C), L-, the boundary shell (C.3), 2LPT (Eqs. 5-6) and the
 * colouring (A.1).  Shared accumulations use FP32 atomics, so results can differ in the last
 * bits between calls.  A position loss must be smooth across the periodic wrap of x (for
 * example a loss of a periodic field sampled at x, as the final density is).
 * Errors: INVALID_ARG (lam_w NULL, or both cotangents NULL); STATE without a checkpointed
 * forward run, or after a scola_lpt_fields, scola_setup_boxes or scola_tcola call that
 * replaced its state.
 */
scola_status scola_backward(scola_ctx *ctx, const float *lam_x_dev, const float *lam_p_dev, float *lam_w_dev);

/*
 * Adjoint of the final density (Sec. 4.1): lam_x = (d delta_final / dx)^T lam_delta for the
 * periodic CIC density of scola_final_density, at the given positions.  Composed with
 * scola_backward it differentiates a loss of the final density.  Needs no forward run.
 *   x_dev          device, Np^3 x 3 FP32 positions in [0, L)
 *   lam_delta_dev  device, Np^3 FP32: dLoss/d delta_final
 *   lam_x_dev      device, Np^3 x 3 FP32, receives dLoss/dx
 * Errors: INVALID_ARG (NULL), CUDA.
 */
scola_status scola_density_adjoint(scola_ctx *ctx, const float *x_dev, const float *lam_delta_dev,
                                   float *lam_x_dev);

/*
 * Gradient of a loss of the final density with respect to the white noise for the last
 * checkpointed scola_forward run: scola_density_adjoint at that run's positions followed by
 * scola_backward, in one call (the positions are taken from the library's particle state,
 * so no x buffer is needed; the result is the same).
 *   lam_delta_dev  device, Np^3 FP32: dLoss/d delta_final (periodic CIC of scola_final_density)
 *   lam_w_dev      device, Np^3 FP32, receives dLoss/dw
 * Errors: as scola_backward.
 */
scola_status scola_backward_density(scola_ctx *ctx, const float *lam_delta_dev, float *lam_w_dev);

/*
 * Box density without any allocation.  The paper has no counterpart: this is
 * an interface for callers that cannot allocate device memory at the point
 * where they need a density (for example a service that forbids allocations
 * outside its own memory pool, or a loop that must not call the allocator).
 * It computes the same B^sCOLA cloud-in-cell density as
 * scola_pm_force's delta output for one box, needs no context, and calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *   s_dev      device, 3 x nsc^3 FP32 displacements s = x - q of the box
 *              particles, [component][particle], box-local order
 *              (bi*nsc + bj)*nsc + bk, particle b at q_loc = (b + 1/2) dq
 *   nsc        particles per side of the box (Np,sCOLA)
 *   ng         PM cells per side (Ng >= nsc); ng^3 <= 128^3 = 2,097,152
 *   dq         lattice spacing L / Np [Mpc/h]
 *   delta_dev  device, ng^3 FP32, receives delta = n / nbar - 1 per interior cell
 *   stream     cudaStream_t for the work (NULL = legacy default stream)
 * Scratch: a fixed 16 MiB device array (128^3 64-bit counters) in the
 * library, held by every GPU that loads the library until the process exits.
 * Every call shares it and it keeps the previous call's contents; each call
 * clears the part it uses first.  Calls whose work overlaps on the GPU
 * (different streams or host threads) race on the scratch: serialise them.
 * The first call on each device looks up the scratch's device address with
 * cudaGetSymbolAddress (with that device current).
 * Errors: INVALID_ARG (NULL pointers, ng < nsc, ng^3 above the maximum),
 * CUDA.
 */
scola_status scola_box_density_noalloc(const float *s_dev, int32_t nsc, int32_t ng, double dq,
                                       float *delta_dev, void *stream);

/*
 * Self-test of the fixed-point conversions of the CIC deposits (the paper has
 * no counterpart).  The deposits convert each FP32 weight w in [0, 1] to the
 * 64-bit integer round(w 2^32) and the summed counts back to FP32 with 32-bit
 * instructions only; this runs those forms and CUDA's direct 64-bit
 * conversions on n generated inputs (weights in [0, 1] including 0, 1 and
 * values near both ends; counts of every magnitude and exact rounding ties)
 * on the current device and counts the results that differ in any bit.
 *   n           number of inputs (>= 0)
 *   seed        input generator seed
 *   mismatches  host, receives the count (0 means bit-identical)
 * Synchronous.  Errors: INVALID_ARG (NULL, n < 0), OOM, CUDA.
 */
scola_status scola_selftest_conversions(int64_t n, uint64_t seed, int64_t *mismatches);

/*
 * Binned power spectrum of a field on the N^3 LPT grid (Sec. 4.2, Eq. 24), with the
 * normalisation P(k) = L^3 <|DFT delta|^2> / N^6 over the modes of each bin (the DFT
 * unnormalised, every mode of the full spectrum counted once).
 *   delta_dev  device, N^3 FP32 field (k fastest), e.g. from scola_final_density;
 *              not modified
 *   nbins      1 .. 2048
 *   edges      host, nbins + 1 increasing FP64 edges [h/Mpc]; bin b holds
 *              edges[b] <= |k| < edges[b+1], |k| = 2 pi / L |n| with n the wrapped
 *              integer wavenumbers
 *   k_mean, pk host, nbins FP64: mean |k| and P(k) of each bin (NaN for empty bins)
 *   n_modes    host, nbins: modes per bin
 * FP32 transform, FP64 sums in a fixed order (deterministic).  Synchronous.
 * Errors: INVALID_ARG (NULL, nbins out of range, edges not increasing), OOM, CUDA.
 */
scola_status scola_power_spectrum(scola_ctx *ctx, const float *delta_dev, int32_t nbins, const double *edges,
                                  double *k_mean, double *pk, int64_t *n_modes);

/*
 * Mass drop and escapes of given box-particle displacements (Sec. 3.4.1-3.4.2), per box:
 *   s_dev      device, 3 x P displacements in the layout of scola_pm_force
 *   deposited  host, nboxes: the CIC weight the box's particles leave inside its interior
 *              mesh (B^sCOLA keeps it and drops the rest; Np,sCOLA^3 minus it is the
 *              mass drop), summed as 2^-32 fixed-point integers (deterministic)
 *   escaped    host, nboxes: particles whose mesh coordinate lies outside
 *              [-N_ghost, Ng + N_ghost - 1] on some axis (the interpolation clamps them)
 *   nboxes     the context's box count
 * One batch only (UNSUPPORTED otherwise).  Synchronous.
 * Errors: INVALID_ARG (NULL, nboxes), UNSUPPORTED, OOM, CUDA.
 */
scola_status scola_box_mass(scola_ctx *ctx, const float *s_dev, double *deposited, int32_t *escaped,
                            int32_t nboxes);

/*
 * Seeded white noise on the N^3 LPT grid (Sec. 3.1, step A.1), generated on the device:
 * Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC11 2011) with key (seed mod 2^32,
 * seed div 2^32); cell i (flat index, k fastest) takes word i % 4 of counter block
 * (i / 4 mod 2^32, i / 4 div 2^32, 0, 0); a word x gives the uniform
 * (floor(x / 2^8) + 1/2) 2^-24, and words (0, 1), (2, 3) give two standard normals each by
 * Box-Muller, sqrt(-2 ln u0) (cos, sin)(2 pi u1), in FP32.  Deterministic for a seed.
 *   w_dev  device, N^3 floats (caller-owned), written on the context stream
 * An alternative to passing any caller-made w to scola_forward.
 * Errors: INVALID_ARG (NULL), CUDA.
 */
scola_status scola_generate_white_noise(scola_ctx *ctx, uint64_t seed, float *w_dev);

/*
 * The periodic full-box tCOLA run (Sec. 2.2; the monolithic simulation that sCOLA
 * approximates, Sec. 4): initial conditions and LPT as scola_forward, then all Np^3
 * particles evolved with the same KDK factors on one periodic PM grid of mesh_ratio * Np
 * cells per side (cells centred at (c + 1/2) dg, dg = L / (mesh_ratio Np)): periodic CIC
 * deposit (2^-32 fixed point, deterministic), FFT Poisson solve with the FDA-2 Laplacian
 * symbol (k = 0 removed), FDA-2 central gradient and periodic CIC interpolation.
 *   w_dev  device, Np^3 white noise (as scola_forward)
 *   x_dev  device, Np^3 x 3 final positions in [0, L), global-id order
 *   p_dev  device, Np^3 x 3 final momenta (L+ applied), global-id order
 * Every particle is written.  FP32 fields and particles; the library's own shared-memory
 * FFTs (power-of-two grids directly, others by Bluestein's chirp transform).
 * Errors: INVALID_ARG (NULL), UNSUPPORTED (fda_order != 2, or mesh_ratio Np outside
 * 2 .. 1024), OOM, CUDA.
 */
scola_status scola_tcola(scola_ctx *ctx, const float *w_dev, float *x_dev, float *p_dev);

scola_status scola_get_stats(const scola_ctx *ctx, scola_stats *out);
const char *scola_status_string(scola_status status);
const char *scola_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SCOLA_H */
