/*
 * sweep.h -- C ABI of the GB300 transport-sweep library (libsweep.so).
 *
 * The library solves the steady, isotropically scattering radiative transfer
 * equation (Peter et al. 2022, Sec. 2.2, Eq. radiativeTransfer) by discrete
 * ordinates on an unstructured (Voronoi) mesh with the Sweep method:
 *   - per direction, a face is upwind/downwind by the sign of n_f.Omega
 *     (Sec. 2.5; Appendix A, Eq. downwindDefinition); an exact zero carries no flux;
 *   - the dependency graph is ordered topologically (Sec. 2.3) into wavefront levels;
 *   - each cell is solved in that order with transport scheme (a) of Sec. 2.6,
 *       (P_c + kappa_t,c V_c) I_c = eps_c/(4 pi) + kappa_s,c V_c J_c + sum_in |a_f| I_up(f),
 *     a_f = A_f n_f.Omega, P_c = sum of a_f over the cell's outflow faces;
 *   - the scattering source iteration (Alg. 1) and the periodic-boundary
 *     iteration (Sec. 2.7, Eq. relativeErrorPbc) run around the sweep.
 * Outputs are the mean intensity J = (1/4pi) sum_d w_d I_d and the absorbed photon
 * rate Gamma = kappa_a V sum_d w_d I_d per cell and frequency group (Sec. 3.2).
 *
 * Conventions
 *   - All calls return a sweep_status and never abort. Outputs are written on
 *     SWEEP_OK and SWEEP_NOT_CONVERGED. The context stays usable after every
 *     error except SWEEP_ERR_CUDA (then destroy it).
 *   - Plain (non-_dev) calls take HOST pointers; the caller owns them and they are
 *     copied during the call (the library keeps no caller pointer).
 *     _dev calls take DEVICE pointers valid on the context's stream; they are read
 *     or written in stream order and the call returns after the work is queued,
 *     except where a convergence decision needs a device-to-host read.
 *   - Array layouts are row-major, C order. Cell arrays are [n_cells]; per-group
 *     arrays are [n_cells][n_groups].
 *   - One context drives one GPU and one CUDA stream. Calls on one context must
 *     not overlap (the context is not thread-safe).
 */
#ifndef SWEEP_H
#define SWEEP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sweep_ctx sweep_ctx; /* opaque; owns every device buffer it allocates */

typedef enum {
    SWEEP_OK = 0,
    SWEEP_ERR_INVALID_ARG = 1, /* bad size, index, flag, value or missing prior set_* call */
    SWEEP_ERR_CYCLE = 2,       /* a direction's dependency graph is cyclic (no topological order, Sec. 2.3) */
    SWEEP_NOT_CONVERGED = 3,   /* an iteration hit its maximum count; outputs are still written */
    SWEEP_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up; outputs are not valid */
    SWEEP_ERR_OOM = 5,         /* device allocation failed */
    SWEEP_ERR_CUDA = 6         /* any other CUDA error; destroy the context */
} sweep_status;

enum { SWEEP_FACE_BOUNDARY = 1, SWEEP_FACE_PERIODIC = 2 };

/* Schedules of the batched sweep kernel. */
enum {
    SWEEP_SCHED_AUTO = 0,     /* pick by a one-time timing of LEVEL vs DATAFLOW per context */
    SWEEP_SCHED_LEVEL = 1,    /* persistent kernel, grid barrier between wavefront levels */
    SWEEP_SCHED_DATAFLOW = 2, /* persistent kernel, no barriers: each task waits (bounded) for its upwind values */
    SWEEP_SCHED_PLAIN = 3     /* plain FP64 path: one kernel launch per (direction, level), no batching */
};

/* Absorption laws of the cell update (transport scheme (a) of Sec. 2.6, outflow = non-absorbed inflow
 * plus source; F_in = the inflow flux, P = the projected outflow area, tau = kappa_t V / P):
 *   BALANCE: (P + kappa_t V) I = q + F_in, and J is formed from I;
 *   EXP:     P I = exp(-tau) F_in + q (the source leaves unattenuated), and J is formed from the
 *            cell-mean intensity (F_in / P)(1 - exp(-tau)) / tau, so that kappa_t V times it is the
 *            removed flux; with kappa_a = 0 the scattered fraction is 1 - exp(-kappa_s V / P), the
 *            scattering law of Sec. 3.3. Forward solves only (the adjoint takes BALANCE). In FP32 EXP
 *            runs over the packed operator (1, 2 or 4 groups; otherwise, and in FP64, in the kernels that
 *            read the mesh rows), on the DATAFLOW schedule when the schedule is AUTO (no autotuning),
 *            and keeps one more [D][N][G] array. */
enum { SWEEP_LAW_BALANCE = 0, SWEEP_LAW_EXP = 1 };

typedef struct {
    int32_t precision;    /* 32: FP32 intensities, FP64 tallies and norms; 64: FP64 throughout */
    int32_t law;          /* SWEEP_LAW_BALANCE (default) or SWEEP_LAW_EXP */
    int32_t schedule;     /* SWEEP_SCHED_*; SWEEP_SCHED_PLAIN implies precision 64 */
    int32_t max_it_scat;  /* source iteration (Alg. 1): maximum sweeps per periodic iteration */
    double tol_scat;      /* stop when max_c |J_new - J_old| / J_new <= tol_scat (0/0 counts as converged) */
    int32_t max_it_pbc;   /* periodic iteration (Sec. 2.7): maximum outer iterations */
    int32_t warm_start;   /* 1: start the periodic iteration from the previous solve's intensities (Sec. 2.7) */
    double tol_pbc;       /* stop when max_i |E_i| < tol_pbc, Eq. relativeErrorPbc */
    int32_t dir_batch;    /* adjoint: directions per recompute batch (0 = all directions at once) */
    int32_t relevel;      /* 1: redo classification and levelisation even if cached for this mesh+directions */
    int32_t block_threads;/* threads per block of the batched sweep (0 = autotuned) */
    int32_t use_graph;    /* 1 (default): run the periodic iteration or the source iteration as CUDA graphs, each
                             distinct iteration captured once per solve and replayed (not with both loops
                             nested, the plain schedule or debug_stall, or when capture is refused: host loop) */
    int64_t spin_budget;  /* bound on each device-side wait, in polls (0 = default, about 1 s) */
    int32_t debug_stall;  /* TEST ONLY: 1 makes the first sweep task wait on a word nothing writes */
    int32_t lanes_per_task; /* lanes cooperating on one task in the batched sweep: 1..16, a power of 2 (0 = autotuned);
                               over the assembled operator 2, 4 or 8 (1 runs as 2), and 16 = 8 lanes per task
                               with two tasks per lane group (one group, dataflow schedule; else as 8) */
    int32_t geometry_only;  /* 1: the FP32 sweep reads the mesh every sweep instead of the assembled operator */
    int32_t blocks_per_sm;  /* resident blocks per SM of the batched sweep (0 = autotuned / maximum) */
    int32_t fused_loops;    /* 1: with both scattering and periodic faces, fuse the two loops as Sec. 2.7 suggests:
                               one source-iteration sweep per periodic iteration, J carried over between periodic
                               iterations, stop when both changes are below tol_scat and tol_pbc (at most max_it_pbc
                               sweeps). Same fixed point as the nested loops (0, default), far fewer sweeps.
                               Ignored unless both loops are on. */
    int32_t op_format;      /* SWEEP_OP_*: form of the assembled operator of the FP32 forward sweep */
    int32_t packets_per_step; /* packed operator: packets a warp takes per step, 1 or 2 (0 = autotuned) */
    int32_t transport;      /* transport scheme of Sec. 2.6: 0 = scheme (a), the outflow split over all outflow faces
                               in proportion to A_f n_f.Omega; n in 1..8 = scheme (b), direction-conserving transport:
                               each cell hands its outflow P_c I_c in equal parts to the n outflow faces whose outward
                               normal is most nearly along Omega (largest n.Omega in FP64, ties to the lower face
                               index), or to all its outflow faces if it has fewer; the dependency graph keeps only
                               those faces. Boundary inflow enters as in scheme (a); a chosen vacuum face lets its
                               part escape, a chosen periodic face passes it to the partner. Rows of at most 64 face
                               sides; forward solves only (the adjoint takes scheme (a)). */
} sweep_opts;

/* Forms of the assembled transport operator (the rows of L_Omega, Sec. 2.3, built once per
 * levelisation and streamed by every FP32 sweep of the solve; the EXP law and scheme (b) take PACKETS
 * only, and the FP32 adjoint streams a packed transposed operator, the rows of L_Omega^T with the
 * levels in reverse order, for 2G = 2 or 4 split groups):
 *   AUTO:    PACKETS where they apply (1, 2 or 4 groups, n_cells x n_dir <= 2^31, lanes_per_task 0),
 *            else LINES;
 *   LINES:   one 128-byte line per task (header + 14 entry slots), lanes_per_task lanes per task;
 *   PACKETS: tasks packed back to back, within a wavefront level, into 512-byte warp packets (two
 *            8-byte slots per lane: the task's inflow entries, then its header), so that no entry slot
 *            of a warp step is empty and every lane gathers; falls back to LINES where it does not apply. */
enum { SWEEP_OP_AUTO = 0, SWEEP_OP_LINES = 1, SWEEP_OP_PACKETS = 2 };

typedef struct {
    int32_t it_scat, it_pbc;   /* sweeps done in the source iteration (total) and periodic iterations */
    int32_t n_sweeps;          /* sweeps of all directions done by the solve */
    int32_t depth_max;         /* largest critical-path depth (levels) over directions */
    double depth_mean;         /* mean depth over directions */
    double res_scat, res_pbc;  /* final residuals (max norm); res_pbc_mean = mean of |E_i| */
    double res_pbc_mean;
    double emitted, injected, absorbed, escaped; /* photons/s over all cells and groups (FP64) */
    double defect;             /* (emitted + injected - absorbed - escaped) / (emitted + injected) */
    double t_ms[8];            /* 0 classify, 1 levelise, 2 sweeps, 3 tallies+updates, 4 total, 5 operator
                                  assembly, 6 (adjoint) the transposed sweeps within 2 (CUDA events) */
    double updates;            /* cell x direction x group updates done by all sweeps */
    double updates_per_s;      /* updates / (t_ms[4] / 1000) */
    int32_t sweep_launches;    /* batched-sweep kernel launches timed in t_ms[2] */
    int32_t schedule_used;     /* SWEEP_SCHED_* that ran */
    int32_t kernel_launches;   /* all kernels this call launched (including the autotuner's) */
    int32_t lanes_used;        /* lanes per task of the batched sweep that ran (packed operator: 32 x packets per step) */
    int32_t threads_used;      /* threads per block of the batched sweep that ran */
    int32_t blocks_per_sm_used;/* resident blocks per SM it was launched with (0 = maximum) */
    int32_t kernel_used;       /* SWEEP_KERNEL_* form of the batched sweep that ran last */
    int32_t graph_used;        /* 1: the iterations ran as CUDA graphs */
} sweep_stats;

/* Forms of the batched sweep kernel (sweep_stats.kernel_used). */
enum {
    SWEEP_KERNEL_NONE = 0,
    SWEEP_KERNEL_PLAIN = 1,          /* one launch per (direction, level), FP64 */
    SWEEP_KERNEL_GEOMETRY = 2,       /* lane groups reading the mesh rows (FP64; FP32 adjoint or EXP without packets) */
    SWEEP_KERNEL_RECORDS = 3,        /* FP32 forward, lane groups over task records and mesh rows */
    SWEEP_KERNEL_OPERATOR = 4,       /* FP32 forward over the assembled operator, lane groups */
    SWEEP_KERNEL_OPERATOR_LEAN = 5,  /* the same, one group and 8 lanes per task, dataflow schedule */
    SWEEP_KERNEL_OPERATOR_PAIR = 6,  /* the same with two tasks per 8-lane group per step */
    SWEEP_KERNEL_PACKED = 7          /* FP32 over the packed operator, forward (BALANCE or EXP) or transposed
                                        (whole warps per packet of tasks) */
};

/* Fill *opts with defaults: precision 32, AUTO schedule, tolerances 1e-6, 100 iterations. */
void sweep_default_opts(sweep_opts* opts);

/* Create a context on CUDA device `device`, issuing all work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). */
sweep_status sweep_create(sweep_ctx** ctx, int device, void* cuda_stream);
sweep_status sweep_destroy(sweep_ctx* ctx);

/* The mesh (Sec. 2.5: cells and their neighbours; Appendix A: face normals).
 *   volume[n_cells]          > 0
 *   face_cells[n_faces][2]   (c0, c1); c1 = -1 on a box-boundary face (flag BOUNDARY);
 *                            with flag PERIODIC, c1 is the partner cell across the box
 *                            (c1 == c0 allowed); faces are stored once
 *   area[n_faces]            >= 0
 *   normal[n_faces][3]       unit (|n| = 1 +- 1e-9), pointing from c0 towards c1
 *                            (outward from c0 on boundary faces)
 *   flags[n_faces]           SWEEP_FACE_BOUNDARY | SWEEP_FACE_PERIODIC (not both)
 *   n_meshes, mesh_cell_offset[n_meshes+1]: independent meshes concatenated in one
 *                            index space (faces must not cross meshes); NULL = one mesh.
 * Limits: n_cells < 2^30, sum of face sides < 2^32. Invalidates material and cached levels.
 * Errors: SWEEP_ERR_INVALID_ARG (nothing is kept), SWEEP_ERR_OOM. */
sweep_status sweep_set_mesh(sweep_ctx* ctx, int64_t n_cells, const double* volume, int64_t n_faces,
                            const int32_t* face_cells, const double* area, const double* normal,
                            const uint8_t* flags, int32_t n_meshes, const int64_t* mesh_cell_offset);

/* The discrete-ordinates direction set (Sec. 2.2; solid angle 4pi/N_dir per bin, Sec. 2.6).
 *   omega[n_dir][3] unit vectors, weight[n_dir] > 0 with sum = 4pi (relative 1e-12).
 * 1 <= n_dir <= 1024, and n_cells * 2^ceil(log2 n_dir) <= 2^32.
 * Invalidates cached levels. Errors: SWEEP_ERR_INVALID_ARG. */
sweep_status sweep_set_directions(sweep_ctx* ctx, int32_t n_dir, const double* omega, const double* weight);

/* Material of the current mesh (Eq. radiativeTransfer), per cell and group, 1 <= n_groups <= 8:
 *   kappa_abs[n_cells][G]   absorption coefficient (>= 0, finite)
 *   kappa_scat[n_cells][G]  isotropic scattering coefficient, or NULL = none
 *   emissivity[n_cells][G]  photons/s emitted by the cell, isotropically (>= 0)
 *   boundary_inflow[n_boundary_faces][G]  isotropic intensity entering through each
 *                           boundary face (in face order), or NULL = vacuum (I = 0, Sec. 2.5)
 * Errors: SWEEP_ERR_INVALID_ARG (no mesh, bad value). */
sweep_status sweep_set_material(sweep_ctx* ctx, int32_t n_groups, const double* kappa_abs,
                                const double* kappa_scat, const double* emissivity,
                                const double* boundary_inflow);
/* Same, with device pointers (values are not range-checked; NaN/negative inputs give undefined results). */
sweep_status sweep_set_material_dev(sweep_ctx* ctx, int32_t n_groups, const double* kappa_abs,
                                    const double* kappa_scat, const double* emissivity,
                                    const double* boundary_inflow);

/* Solve: classification + levelisation (cached per mesh and direction set), then the
 * periodic iteration (outer, Sec. 2.7) around the source iteration (inner, Alg. 1)
 * around the batched sweep. Writes mean_intensity and absorbed_rate [n_cells][G]
 * (either may be NULL) and *stats (may be NULL).
 * Errors: INVALID_ARG (missing set_*), CYCLE, TIMEOUT, OOM, CUDA; NOT_CONVERGED with outputs. */
sweep_status sweep_solve(sweep_ctx* ctx, const sweep_opts* opts, double* mean_intensity, double* absorbed_rate,
                         sweep_stats* stats);
sweep_status sweep_solve_dev(sweep_ctx* ctx, const sweep_opts* opts, double* mean_intensity,
                             double* absorbed_rate, sweep_stats* stats);

/* Wavefront level of every cell for direction `dir` (0 = no upwind cell, else 1 + the
 * largest level of its upwind cells: the longest dependency path, Sec. 2.3) and the
 * direction's depth (1 + largest level), in the dependency graph of the transport scheme the
 * cached levels were made for (that of the last solve; scheme (a) when nothing is cached).
 * Classifies and levelises if not cached. level[n_cells] host pointer. Errors: INVALID_ARG, CYCLE. */
sweep_status sweep_levels(sweep_ctx* ctx, int32_t dir, int32_t* level, int32_t* depth);

/* Intensity of direction `dir` from the last solve's final sweep, as FP64, [n_cells][G]
 * host pointer. Errors: INVALID_ARG (no solve yet or bad dir). */
sweep_status sweep_intensity(sweep_ctx* ctx, int32_t dir, double* intensity);

/* Rotation of the direction set between substeps (Sec. 2.6, the rotation paragraph): a radiative-
 * transfer step may be split into N_rot substeps, each with the sources reduced by 1/N_rot, the
 * directions rotated after every substep to Omega'_i = R Omega_i (R a rotation, e.g. R_z(phi) R_y(theta)
 * with randomly drawn spherical angles). Angle-dependent state is carried over by
 *   I(Omega'_i) = sum_j c_ij I(Omega_j),  c_ij = dS_ij / dS_i,
 * dS_ij the solid angle that the bin of new direction i shares with the bin of old direction j (a bin:
 * the part of the unit sphere nearer to its direction than to any other of its set; nearest by the
 * largest ((px Ox) + (py Oy)) + (pz Oz) in FP64, ties to the lower index) and dS_i = sum_j dS_ij,
 * taken by a quadrature of n_quad equal-weight points of a Fibonacci sphere
 * (z_m = 1 - (2m+1)/n_quad, phi_m = m pi (3 - sqrt 5)).
 *   rotation[3][3]  HOST pointer, row-major; orthonormal with determinant +1 (within 1e-12)
 *   n_quad          quadrature points, 1 .. 2^26 (0 = 2^16)
 * The context's directions become Omega'_i = ((R_k0 x + R_k1 y) + R_k2 z) (weights unchanged; cached
 * levels and operators are rebuilt by the next solve), and the intensities of the last solve are
 * remapped, so that a following solve with warm_start = 1 starts its periodic iteration from them.
 * The caller scales the sources by 1/N_rot and sums the substeps' J and Gamma.
 * Errors: INVALID_ARG (no directions, bad rotation or n_quad), OOM, CUDA. */
sweep_status sweep_rotate_directions(sweep_ctx* ctx, const double* rotation, int64_t n_quad);

/* Adjoint (transpose) of the sweep for a loss L(J, Gamma). For each direction it solves
 * L_Omega^T lambda = g, g_c = w_d (dL/dGamma_c kappa_a,c V_c + dL/dJ_c / 4pi), as a sweep
 * in reversed level order, and accumulates in FP64
 *   dL/dkappa_a,c = sum_d V_c I_c,d (w_d dL/dGamma_c - lambda_c,d),  dL/deps_c = sum_d lambda_c,d / 4pi.
 * Without scattering and periodic faces the forward intensities are recomputed per batch of
 * opts->dir_batch directions instead of stored. With scattering (Alg. 1) or periodic faces
 * (Sec. 2.7) the forward state is the solve itself (sweep_solve with the same opts, both
 * iterations to their tolerances), and lambda solves the transpose of the coupled system,
 *   L_Omega^T lambda_d = g_d + P_d^T lambda_d + w_d kappa_s,c V_c mu_c / 4pi,  mu_c = sum_d lambda_c,d,
 * P_d the periodic inflow coupling, by one transposed iteration that lags both couplings by a
 * pass: mu and the previous pass's lambda start at 0, each pass sweeps every direction in
 * reversed level order reading the partner's lambda of the previous pass across periodic outflow
 * sides, and the iteration stops when max |change of mu| <= tol_scat max |mu| or after
 * max_it_scat passes. grad_kappa_scat (or NULL) receives
 *   dL/dkappa_s,c = sum_d V_c lambda_c,d (J_c - I_c,d).
 * With scattering, periodic faces or grad_kappa_scat, dir_batch is ignored.
 * dl_dJ, dl_dGamma [n_cells][G] (either may be NULL = zero); outputs [n_cells][G], host pointers
 * for sweep_adjoint and device pointers for sweep_adjoint_dev. stats (or NULL): it_scat = forward
 * sweeps, it_pbc = transposed passes, res_scat / res_pbc = their last relative changes. The solve
 * buffers (sweep_intensity) then hold the forward state.
 * Errors: INVALID_ARG (more than 4 groups, missing set_*), CYCLE, TIMEOUT, OOM, CUDA;
 * NOT_CONVERGED (gradients still written) when the forward solve or the transposed iteration hit
 * its maximum. */
sweep_status sweep_adjoint(sweep_ctx* ctx, const sweep_opts* opts, const double* dl_dJ, const double* dl_dGamma,
                           double* grad_kappa_abs, double* grad_emissivity, double* grad_kappa_scat,
                           sweep_stats* stats);
sweep_status sweep_adjoint_dev(sweep_ctx* ctx, const sweep_opts* opts, const double* dl_dJ,
                               const double* dl_dGamma, double* grad_kappa_abs, double* grad_emissivity,
                               double* grad_kappa_scat, sweep_stats* stats);

/* Wavefront levels of one direction without any device allocation. The paper has no counterpart:
 * this serves callers that cannot allocate GPU memory where they need a sweep order (a fixed
 * device-memory budget such as an arena or pool that hands out no new blocks, or memory nearly
 * exhausted by another component, where cudaMalloc would fail or stall the device).
 *   device, cuda_stream    the GPU and stream to run on (NULL stream = legacy default stream)
 *   face_cells[n_faces][2], normal[n_faces][3], flags[n_faces]
 *                          DEVICE pointers, the mesh faces as for sweep_set_mesh (the cell indices of
 *                          interior faces are checked on the device: INVALID_ARG, nothing out of range
 *                          is touched; normals and flags are not validated)
 *   omega[3]               HOST pointer, the direction
 *   level[n_cells]         DEVICE output: level of every cell (as sweep_levels)
 *   depth                  HOST output: 1 + the largest level
 * Limit: 1 <= n_cells <= 65536; larger meshes are rejected with SWEEP_ERR_INVALID_ARG before any
 * GPU work. The working memory is one static device array (65536 counters plus a control block,
 * 256 KB) that every GPU loading the library holds until exit; every call shares it and clears
 * what must start at zero, so calls whose GPU work overlaps (other host threads, other streams)
 * race and give wrong results. Every call looks up the array's device address (the first call on a
 * device also loads the library's device code there, a one-time set-up; make that first call before
 * any stream capture); the lookup allocates nothing. The call returns after the result is on the
 * device (it synchronizes the stream). Errors: INVALID_ARG (sizes, null pointers, device, a face
 * cell index outside [0, n_cells)), CYCLE, TIMEOUT (a bounded wait gave up), CUDA. */
sweep_status sweep_levels_noalloc(int device, void* cuda_stream, int64_t n_cells, int64_t n_faces,
                                  const int32_t* face_cells, const double* normal, const uint8_t* flags,
                                  const double* omega, int32_t* level, int32_t* depth);

/* Static description of a status code; sweep_last_error gives the context's last detailed message. */
const char* sweep_status_string(sweep_status status);
const char* sweep_last_error(const sweep_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SWEEP_H */
