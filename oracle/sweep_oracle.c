/*
 * sweep_oracle.c -- plain, slow FP64 CPU oracle of the discrete-ordinates transport
 * sweep (Peter et al. 2022, "The Sweep Method for radiative transfer in Arepo").
 *
 * TEST INFRASTRUCTURE ONLY. This file is the reference the CUDA path is checked
 * against. Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the product path never calls it. It shares no code,
 * header or constant with the CUDA library.
 *
 * Build with -ffp-contract=off: every dot product is ((x*x') + (y*y')) + (z*z')
 * with separately rounded products, so classification signs are reproducible.
 *
 * What it computes, step by step, in the paper's order:
 *   O1 classify   -- a neighbour is downwind when n.Omega > 0 (Sec. 2.5; Appendix A,
 *                    Eq. downwindDefinition). An exact zero is neither upwind nor
 *                    downwind and carries no flux (reading of the "upwind otherwise"
 *                    rule that keeps the dependency graph acyclic).
 *   O2 count+Kahn -- Alg. 2 (single-core sweep): count upwind fluxes n(c,Omega),
 *                    queue the tasks with n = 0, solve, decrement downwind counts.
 *                    The level of a cell is 0 without upwind cells, else
 *                    1 + max(level of upwind cells) (longest path, Sec. 2.3).
 *   O3 cell update-- transport scheme (a) of Sec. 2.6 (Eq. for F_i): the total
 *                    outflow F leaves through downwind face i in proportion to
 *                    A_i (n_i.Omega). Written as a cell balance,
 *                      (P_c + kappa_t V) I_c = q_c + sum_in |a_f| I_up(f),
 *                    a_f = A_f n_f.Omega, P_c = sum over outflow faces of a_f,
 *                    q_c = eps_c/(4 pi) + kappa_s V J_c  (Eq. radiativeTransfer
 *                    discretised with isotropic emission and scattering).
 *   O4 tallies    -- J = (1/4pi) sum_d w_d I_d; absorbed rate
 *                    Gamma = kappa_a V sum_d w_d I_d (photon rate R of Sec. 3.2 up to
 *                    the 13.6 eV factor); escaped and injected boundary fluxes.
 *   O5 scattering -- Alg. 1 (source iteration) with I^0 = 0; stop when the relative
 *                    change of J is below tol in every cell (Sec. 2.3 criterion,
 *                    applied to the mean intensity).
 *   O6 periodic   -- Sec. 2.7: flux leaving through a periodic face enters the
 *                    partner cell as a source in the next sweep; stop when
 *                    max_i |E_i| < tol, E_i = (j^n - j^(n-1)) / (j^n + j^(n-1))
 *                    (Eq. relativeErrorPbc) or after max_it sweeps.
 *   O7 nesting    -- periodic iteration outside, source iteration inside
 *                    (cost n_pbc * n_scat, Sec. 2.7).
 *   O9 adjoint    -- transpose of the O3 system per direction, solved as a sweep in
 *                    reversed topological order; gradients of a loss of J and Gamma
 *                    with respect to kappa_a and eps.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define FOURPI (4.0 * 3.14159265358979323846)

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_CYCLE = 2, OR_NOT_CONVERGED = 3, OR_ERR_MEM = 5 };
enum { OR_FACE_BOUNDARY = 1, OR_FACE_PERIODIC = 2 };
enum { OR_LAW_BALANCE = 0, OR_LAW_EXP = 1 };

typedef struct {
    /* problem (caller-owned) */
    int64_t n_cells, n_faces;
    const double* volume;
    const int32_t* face_cells; /* [F][2] */
    const double* area;
    const double* normal; /* [F][3] */
    const uint8_t* flags;
    int32_t n_dir;
    const double* omega; /* [D][3] */
    const double* weight;
    int32_t n_groups;
    const double* kappa_abs;  /* [N][G] */
    const double* kappa_scat; /* [N][G] or NULL */
    const double* emissivity; /* [N][G] */
    const double* bc_inflow;  /* [n_boundary_faces][G] or NULL */
    int law;                  /* OR_LAW_BALANCE or OR_LAW_EXP (forward sweeps only) */
    int dc_n;                 /* 0: scheme (a); n > 0: direction-conserving transport to n neighbours */
    double* mean;             /* EXP: [D][N][G] cell-mean intensity of the last sweep (solver-owned) */
    /* derived: per-cell list of face sides */
    int64_t* side_start; /* [N+1] */
    int64_t* side_face;  /* face index */
    int8_t* side_sign;   /* +1 if the cell is c0 (outward normal = n), -1 if c1 */
    int64_t* bc_index;   /* [F] boundary face ordinal, -1 otherwise */
    int64_t* face_side;  /* [F][2] side index of the face in c0's and in c1's list (-1 if none) */
} problem;

/* O1: the classification dot product, fixed order, no fused multiply-add */
static double face_dot(const double* n, const double* om) {
    double x = n[0] * om[0];
    double y = n[1] * om[1];
    double z = n[2] * om[2];
    return (x + y) + z;
}

static int build_sides(problem* p) {
    int64_t N = p->n_cells, F = p->n_faces;
    p->side_start = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
    p->bc_index = (int64_t*)malloc(sizeof(int64_t) * (size_t)(F > 0 ? F : 1));
    if (!p->side_start || !p->bc_index) return OR_ERR_MEM;
    int64_t nb = 0;
    for (int64_t f = 0; f < F; ++f) {
        int32_t c0 = p->face_cells[2 * f], c1 = p->face_cells[2 * f + 1];
        p->side_start[c0 + 1]++;
        if (c1 >= 0) p->side_start[c1 + 1]++;
        p->bc_index[f] = (p->flags[f] & OR_FACE_BOUNDARY) ? nb++ : -1;
    }
    for (int64_t c = 0; c < N; ++c) p->side_start[c + 1] += p->side_start[c];
    int64_t S = p->side_start[N];
    p->side_face = (int64_t*)malloc(sizeof(int64_t) * (size_t)(S > 0 ? S : 1));
    p->side_sign = (int8_t*)malloc((size_t)(S > 0 ? S : 1));
    p->face_side = (int64_t*)malloc(sizeof(int64_t) * 2 * (size_t)(F > 0 ? F : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    if (!p->side_face || !p->side_sign || !p->face_side || !fill) { free(fill); return OR_ERR_MEM; }
    for (int64_t c = 0; c < N; ++c) fill[c] = p->side_start[c];
    for (int64_t f = 0; f < F; ++f) {
        int32_t c0 = p->face_cells[2 * f], c1 = p->face_cells[2 * f + 1];
        p->face_side[2 * f] = fill[c0];
        p->face_side[2 * f + 1] = c1 >= 0 ? fill[c1] : -1;
        p->side_face[fill[c0]] = f;
        p->side_sign[fill[c0]++] = 1;
        if (c1 >= 0) {
            p->side_face[fill[c1]] = f;
            p->side_sign[fill[c1]++] = -1;
        }
    }
    free(fill);
    return OR_OK;
}

static void free_sides(problem* p) {
    free(p->side_start);
    free(p->side_face);
    free(p->side_sign);
    free(p->bc_index);
    free(p->face_side);
}

/* cell on the other side of a face side (interior or periodic partner) */
static int32_t other_cell(const problem* p, int64_t f, int sign) {
    return sign > 0 ? p->face_cells[2 * f + 1] : p->face_cells[2 * f];
}

/*
 * Direction-conserving transport (scheme (b) of Sec. 2.6): every cell hands its outflow in equal
 * parts to the dc_n outflow sides whose outward normal is most nearly along Omega (largest
 * n . Omega; on a tie the lower face index), or to all its outflow sides if it has fewer. For one
 * direction (t[f] = n_f . Omega) this marks chosen[k] for every side k and gives share[c] =
 * P_c / n_c, the flux per unit intensity through each chosen side (P_c the projected outflow
 * area, as in scheme (a), n_c the number of chosen sides).
 */
static void dc_choose(const problem* p, const double* t, uint8_t* chosen, double* share) {
    for (int64_t c = 0; c < p->n_cells; ++c) {
        int64_t k0 = p->side_start[c], k1 = p->side_start[c + 1];
        double P = 0.0;
        int n = 0;
        for (int64_t k = k0; k < k1; ++k) {
            chosen[k] = 0;
            int64_t f = p->side_face[k];
            double tout = p->side_sign[k] > 0 ? t[f] : -t[f];
            if (tout > 0.0) P += p->area[f] * tout;
        }
        for (int m = 0; m < p->dc_n; ++m) {
            int64_t best = -1;
            double bt = 0.0;
            for (int64_t k = k0; k < k1; ++k) {
                if (chosen[k]) continue;
                int64_t f = p->side_face[k];
                double tout = p->side_sign[k] > 0 ? t[f] : -t[f];
                if (!(tout > 0.0)) continue;
                if (best < 0 || tout > bt || (tout == bt && f < p->side_face[best])) { best = k; bt = tout; }
            }
            if (best < 0) break;
            chosen[best] = 1;
            ++n;
        }
        share[c] = n > 0 ? P / n : 0.0;
    }
}

/* flux per unit upwind intensity through face f from its upwind cell u (side ku of u): |a_f| in
 * scheme (a); share[u] if the side is one of u's chosen ones, else 0, in scheme (b) */
static double face_weight(const problem* p, const uint8_t* chosen, const double* share, int64_t f, double tabs,
                          int32_t u, int64_t ku) {
    if (!chosen) return p->area[f] * tabs;
    return chosen[ku] ? share[u] : 0.0;
}

/*
 * Alg. 2 for one direction: the Kahn task queue over cells, with levels.
 * t[f] = n_f . Omega for every face. Returns OR_ERR_CYCLE if tasks remain.
 * If solve != 0 the O3 update is applied to each task as it is dequeued:
 *   forward (reverse = 0): inflow faces have outward t < 0, upwind = across them;
 *   adjoint (reverse = 1): the transposed system; "inflow" is the outflow side.
 */
typedef struct {
    const problem* p;
    const double* t;   /* [F] */
    int reverse;
    const double* src; /* [N][G] source q (forward) or adjoint source g */
    const double* prev; /* [N][G] previous-sweep intensity for periodic inflow, or NULL */
    double* out;       /* [N][G] solution */
    double* mean;      /* [N][G] EXP law: cell-mean intensity, or NULL */
    const uint8_t* chosen; /* [S] scheme (b): the chosen outflow sides of this direction, or NULL */
    const double* share;   /* [N] scheme (b): flux per unit intensity through each chosen side */
    int32_t* level;    /* [N] or NULL */
    int32_t* depth;
    /* scratch */
    int32_t* count;
    int64_t* queue;
} dir_sweep;

static int sweep_one(dir_sweep* s, int solve) {
    const problem* p = s->p;
    int64_t N = p->n_cells;
    int G = p->n_groups;
    /* count upwind fluxes n(c, Omega) over interior, non-periodic faces (scheme (b): the faces the
     * upwind cell hands flux to) */
    for (int64_t c = 0; c < N; ++c) s->count[c] = 0;
    for (int64_t f = 0; f < p->n_faces; ++f) {
        if (p->flags[f] & (OR_FACE_BOUNDARY | OR_FACE_PERIODIC)) continue;
        double t = s->t[f];
        if (s->reverse) t = -t;
        if (t == 0.0) continue;
        if (s->chosen && !s->chosen[p->face_side[2 * f + (t > 0.0 ? 0 : 1)]]) continue;
        if (t > 0.0) s->count[p->face_cells[2 * f + 1]]++;
        else s->count[p->face_cells[2 * f]]++;
    }
    int64_t head = 0, tail = 0;
    for (int64_t c = 0; c < N; ++c) {
        if (s->level) s->level[c] = 0;
        if (s->count[c] == 0) s->queue[tail++] = c;
    }
    int32_t maxlev = -1;
    while (head < tail) {
        int64_t c = s->queue[head++];
        if (s->level && s->level[c] > maxlev) maxlev = s->level[c];
        if (solve) {
            double P = 0.0;
            double acc[64];
            /* BALANCE sums the source first, then the inflows; EXP keeps the inflow F_in apart */
            for (int g = 0; g < G; ++g) acc[g] = s->mean ? 0.0 : s->src[c * G + g];
            for (int64_t k = p->side_start[c]; k < p->side_start[c + 1]; ++k) {
                int64_t f = p->side_face[k];
                int sign = p->side_sign[k];
                double tout = sign > 0 ? s->t[f] : -s->t[f]; /* n_outward . Omega */
                double a = p->area[f] * fabs(tout);
                int inflow = s->reverse ? (tout > 0.0) : (tout < 0.0);
                if (tout > 0.0) P += a; /* P_c: projected outflow area (both directions) */
                if (!inflow || tout == 0.0) continue;
                uint8_t fl = p->flags[f];
                if (fl & OR_FACE_BOUNDARY) {
                    if (!s->reverse && p->bc_inflow) {
                        int64_t b = p->bc_index[f];
                        for (int g = 0; g < G; ++g) acc[g] += a * p->bc_inflow[b * G + g];
                    }
                } else if (fl & OR_FACE_PERIODIC) {
                    /* forward: the partner's intensity of the previous sweep flows in; adjoint: the
                     * transpose, the partner's lambda of the previous pass across the outflow side */
                    if (s->prev) {
                        int32_t up = other_cell(p, f, sign);
                        double w = face_weight(p, s->chosen, s->share, f, fabs(tout), up,
                                               p->face_side[2 * f + (sign > 0 ? 1 : 0)]);
                        for (int g = 0; g < G; ++g) acc[g] += w * s->prev[(int64_t)up * G + g];
                    }
                } else {
                    int32_t up = other_cell(p, f, sign);
                    double w = face_weight(p, s->chosen, s->share, f, fabs(tout), up,
                                           p->face_side[2 * f + (sign > 0 ? 1 : 0)]);
                    for (int g = 0; g < G; ++g) acc[g] += w * s->out[(int64_t)up * G + g];
                }
            }
            for (int g = 0; g < G; ++g) {
                double kt = p->kappa_abs[c * G + g] + (p->kappa_scat ? p->kappa_scat[c * G + g] : 0.0);
                if (!s->mean) {
                    s->out[c * G + g] = acc[g] / (P + kt * p->volume[c]);
                } else if (P > 0.0) {
                    /* EXP: the inflow crosses the mean chord V/P with transmission exp(-tau) and the
                     * cell's own source leaves unattenuated (Sec. 2.6); the cell-mean intensity of
                     * the attenuated inflow is (F_in/P)(1 - exp(-tau))/tau */
                    double q = s->src[c * G + g];
                    double tau = kt * p->volume[c] / P;
                    double f = tau > 0.0 ? -expm1(-tau) / tau : 1.0;
                    s->out[c * G + g] = (exp(-tau) * acc[g] + q) / P;
                    s->mean[c * G + g] = acc[g] / P * f;
                } else {
                    /* no outflow in this direction: everything that enters or is emitted stays */
                    double v = (acc[g] + s->src[c * G + g]) / (kt * p->volume[c]);
                    s->out[c * G + g] = v;
                    s->mean[c * G + g] = v;
                }
            }
        }
        /* release the downwind tasks */
        for (int64_t k = p->side_start[c]; k < p->side_start[c + 1]; ++k) {
            int64_t f = p->side_face[k];
            if (p->flags[f] & (OR_FACE_BOUNDARY | OR_FACE_PERIODIC)) continue;
            if (s->chosen && !s->chosen[k]) continue;
            int sign = p->side_sign[k];
            double tout = sign > 0 ? s->t[f] : -s->t[f];
            if (s->reverse) tout = -tout;
            if (tout > 0.0) {
                int32_t d = other_cell(p, f, sign);
                if (s->level && s->level[d] < s->level[c] + 1) s->level[d] = s->level[c] + 1;
                if (--s->count[d] == 0) s->queue[tail++] = d;
            }
        }
    }
    if (s->depth) *s->depth = maxlev + 1;
    return tail == N ? OR_OK : OR_ERR_CYCLE;
}

static void classify(const problem* p, int32_t d, double* t) {
    for (int64_t f = 0; f < p->n_faces; ++f) t[f] = face_dot(p->normal + 3 * f, p->omega + 3 * d);
}

/* --------------------------------------------------------------------------------------------- */
/* threads over directions */
typedef struct {
    const problem* p;
    int32_t d0, d1;
    int reverse;
    const double* src;    /* [N][G] (shared by all directions) or per-direction if src_stride */
    int64_t src_stride;   /* elements between directions' sources (0 = shared) */
    const double* prev;   /* [D][N][G] or NULL */
    double* out;          /* [D][N][G] */
    int32_t* level;       /* [D][N] or NULL */
    int32_t* depth;       /* [D] */
    int solve;
    int status;
} job;

static void* run_job(void* arg) {
    job* j = (job*)arg;
    const problem* p = j->p;
    int64_t N = p->n_cells, G = p->n_groups;
    double* t = (double*)malloc(sizeof(double) * (size_t)(p->n_faces > 0 ? p->n_faces : 1));
    int32_t* count = (int32_t*)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    int32_t* lev = (int32_t*)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    int64_t S = p->side_start[N];
    uint8_t* chosen = p->dc_n > 0 ? (uint8_t*)malloc((size_t)(S > 0 ? S : 1)) : NULL;
    double* share = p->dc_n > 0 ? (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1)) : NULL;
    j->status = OR_OK;
    if (!t || !count || !queue || !lev || (p->dc_n > 0 && (!chosen || !share))) { j->status = OR_ERR_MEM; goto done; }
    for (int32_t d = j->d0; d < j->d1; ++d) {
        classify(p, d, t);
        if (chosen) dc_choose(p, t, chosen, share);
        dir_sweep s;
        s.p = p;
        s.t = t;
        s.reverse = j->reverse;
        s.src = j->src ? j->src + (int64_t)d * j->src_stride : NULL;
        s.prev = j->prev ? j->prev + (int64_t)d * N * G : NULL;
        s.out = j->out ? j->out + (int64_t)d * N * G : NULL;
        s.mean = (p->law == OR_LAW_EXP && !j->reverse && p->mean) ? p->mean + (int64_t)d * N * G : NULL;
        s.chosen = chosen;
        s.share = share;
        s.level = j->level ? j->level + (int64_t)d * N : lev;
        s.depth = j->depth ? j->depth + d : NULL;
        s.count = count;
        s.queue = queue;
        int rc = sweep_one(&s, j->solve);
        if (rc != OR_OK) { j->status = rc; break; }
    }
done:
    free(t);
    free(count);
    free(queue);
    free(lev);
    free(chosen);
    free(share);
    return NULL;
}

static int run_dirs(const problem* p, int n_threads, int reverse, const double* src, int64_t src_stride,
                    const double* prev, double* out, int32_t* level, int32_t* depth, int solve) {
    int32_t D = p->n_dir;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > D) n_threads = D > 0 ? D : 1;
    job* jobs = (job*)calloc((size_t)n_threads, sizeof(job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return OR_ERR_MEM; }
    for (int i = 0; i < n_threads; ++i) {
        jobs[i].p = p;
        jobs[i].d0 = (int32_t)((int64_t)D * i / n_threads);
        jobs[i].d1 = (int32_t)((int64_t)D * (i + 1) / n_threads);
        jobs[i].reverse = reverse;
        jobs[i].src = src;
        jobs[i].src_stride = src_stride;
        jobs[i].prev = prev;
        jobs[i].out = out;
        jobs[i].level = level;
        jobs[i].depth = depth;
        jobs[i].solve = solve;
    }
    if (n_threads == 1) run_job(&jobs[0]);
    else {
        for (int i = 0; i < n_threads; ++i) pthread_create(&th[i], NULL, run_job, &jobs[i]);
        for (int i = 0; i < n_threads; ++i) pthread_join(th[i], NULL);
    }
    int rc = OR_OK;
    for (int i = 0; i < n_threads; ++i)
        if (jobs[i].status != OR_OK) rc = jobs[i].status;
    free(jobs);
    free(th);
    return rc;
}

static int check_problem(const problem* p) {
    if (p->n_cells < 0 || p->n_faces < 0 || p->n_dir < 1 || p->n_groups < 1 || p->n_groups > 64) return OR_ERR_ARG;
    for (int64_t f = 0; f < p->n_faces; ++f) {
        int32_t c0 = p->face_cells[2 * f], c1 = p->face_cells[2 * f + 1];
        if (c0 < 0 || c0 >= p->n_cells || c1 >= p->n_cells) return OR_ERR_ARG;
        if (c1 < 0 && !(p->flags[f] & OR_FACE_BOUNDARY)) return OR_ERR_ARG;
        if (c1 >= 0 && (p->flags[f] & OR_FACE_BOUNDARY)) return OR_ERR_ARG;
    }
    return OR_OK;
}

/* --------------------------------------------------------------------------------------------- */
/* public entry points (loaded with ctypes by the tests) */

/* O1+O2: levels[d][c] and depth[d] for every direction; OR_ERR_CYCLE if a graph is cyclic.
 * dc_n = 0: the dependency graph of scheme (a) (every interior outflow face); dc_n > 0: that of
 * direction-conserving transport, only the faces each cell hands flux to (dc_choose). */
int oracle_levels(int64_t n_cells, int64_t n_faces, const double* volume, const int32_t* face_cells,
                  const double* area, const double* normal, const uint8_t* flags, int32_t n_dir,
                  const double* omega, int dc_n, int32_t* level, int32_t* depth, int n_threads) {
    if (dc_n < 0) return OR_ERR_ARG;
    problem p;
    memset(&p, 0, sizeof p);
    p.n_cells = n_cells; p.n_faces = n_faces; p.volume = volume; p.face_cells = face_cells;
    p.area = area; p.normal = normal; p.flags = flags; p.n_dir = n_dir; p.omega = omega; p.n_groups = 1;
    p.dc_n = dc_n;
    int rc = check_problem(&p);
    if (rc != OR_OK) return rc;
    rc = build_sides(&p);
    if (rc == OR_OK) rc = run_dirs(&p, n_threads, 0, NULL, 0, NULL, NULL, level, depth, 0);
    free_sides(&p);
    return rc;
}

typedef struct {
    int32_t it_scat, it_pbc;
    double res_scat, res_pbc, res_pbc_mean;
    double emitted, injected, absorbed, escaped, defect;
} oracle_stats;

/* per cell and group: (1/4pi) sum_d w_d I_d */
static void mean_intensity(const problem* p, const double* I, double* J) {
    int64_t N = p->n_cells, G = p->n_groups;
    for (int64_t i = 0; i < N * G; ++i) J[i] = 0.0;
    for (int32_t d = 0; d < p->n_dir; ++d)
        for (int64_t i = 0; i < N * G; ++i) J[i] += p->weight[d] * I[(int64_t)d * N * G + i];
    for (int64_t i = 0; i < N * G; ++i) J[i] /= FOURPI;
}

/* j_c: sum_d w_d sum over periodic inflow faces of c of |a_f| I_prev[partner] */
/* per-direction scratch of scheme (b) for the tallies: the chosen sides and shares of direction d
 * (t: [F] scratch for n . Omega); a no-op in scheme (a) */
typedef struct {
    double* t;
    uint8_t* chosen;
    double* share;
} dc_scratch;

static int dc_scratch_init(const problem* p, dc_scratch* x) {
    memset(x, 0, sizeof *x);
    if (p->dc_n <= 0) return OR_OK;
    int64_t S = p->side_start[p->n_cells];
    x->t = (double*)malloc(sizeof(double) * (size_t)(p->n_faces > 0 ? p->n_faces : 1));
    x->chosen = (uint8_t*)malloc((size_t)(S > 0 ? S : 1));
    x->share = (double*)malloc(sizeof(double) * (size_t)(p->n_cells > 0 ? p->n_cells : 1));
    return (x->t && x->chosen && x->share) ? OR_OK : OR_ERR_MEM;
}

static void dc_scratch_dir(const problem* p, dc_scratch* x, int32_t d) {
    if (!x->chosen) return;
    classify(p, d, x->t);
    dc_choose(p, x->t, x->chosen, x->share);
}

static void dc_scratch_free(dc_scratch* x) {
    free(x->t);
    free(x->chosen);
    free(x->share);
}

static void periodic_source(const problem* p, const double* I, double* j, dc_scratch* x) {
    int64_t N = p->n_cells, G = p->n_groups;
    for (int64_t i = 0; i < N * G; ++i) j[i] = 0.0;
    for (int32_t d = 0; d < p->n_dir; ++d) {
        const double* om = p->omega + 3 * d;
        dc_scratch_dir(p, x, d);
        for (int64_t f = 0; f < p->n_faces; ++f) {
            if (!(p->flags[f] & OR_FACE_PERIODIC)) continue;
            double t = face_dot(p->normal + 3 * f, om);
            if (t == 0.0) continue;
            int32_t c0 = p->face_cells[2 * f], c1 = p->face_cells[2 * f + 1];
            int32_t down = t > 0.0 ? c1 : c0, up = t > 0.0 ? c0 : c1;
            double a = face_weight(p, x->chosen, x->share, f, fabs(t), up, p->face_side[2 * f + (t > 0.0 ? 0 : 1)]);
            for (int g = 0; g < G; ++g)
                j[(int64_t)down * G + g] += p->weight[d] * a * I[(int64_t)d * N * G + (int64_t)up * G + g];
        }
    }
}

/* the field J is taken from: the intensity itself (BALANCE) or the cell mean (EXP) */
static const double* tally_field(const problem* p, const double* I) {
    return p->law == OR_LAW_EXP ? p->mean : I;
}

static void tallies(const problem* p, const double* I, double* J, double* Gam, oracle_stats* st, dc_scratch* x) {
    int64_t N = p->n_cells, G = p->n_groups;
    mean_intensity(p, tally_field(p, I), J);
    double emitted = 0.0, absorbed = 0.0, escaped = 0.0, injected = 0.0, wsum = 0.0;
    for (int32_t d = 0; d < p->n_dir; ++d) wsum += p->weight[d];
    for (int64_t c = 0; c < N; ++c)
        for (int g = 0; g < G; ++g) {
            double ka = p->kappa_abs[c * G + g];
            Gam[c * G + g] = ka * p->volume[c] * FOURPI * J[c * G + g];
            absorbed += Gam[c * G + g];
            emitted += p->emissivity[c * G + g] * wsum / FOURPI;
        }
    for (int32_t d = 0; d < p->n_dir; ++d) {
        const double* om = p->omega + 3 * d;
        dc_scratch_dir(p, x, d);
        for (int64_t f = 0; f < p->n_faces; ++f) {
            if (!(p->flags[f] & OR_FACE_BOUNDARY)) continue;
            double t = face_dot(p->normal + 3 * f, om);
            double a = p->area[f] * fabs(t);
            int32_t c = p->face_cells[2 * f];
            /* scheme (b): a cell's outflow leaves through a vacuum face only if it is a chosen side */
            double aout = t > 0.0 ? face_weight(p, x->chosen, x->share, f, fabs(t), c, p->face_side[2 * f]) : 0.0;
            for (int g = 0; g < G; ++g) {
                if (t > 0.0) escaped += p->weight[d] * aout * I[(int64_t)d * N * G + (int64_t)c * G + g];
                else if (t < 0.0 && p->bc_inflow) injected += p->weight[d] * a * p->bc_inflow[p->bc_index[f] * G + g];
            }
        }
    }
    st->emitted = emitted;
    st->injected = injected;
    st->absorbed = absorbed;
    st->escaped = escaped;
    double in = emitted + injected;
    st->defect = in > 0.0 ? (in - absorbed - escaped) / in : 0.0;
}

/* relative change of the mean intensity, max over cells (0/0 counts as converged) */
static double scat_residual(int64_t n, const double* Jnew, const double* Jold) {
    double r = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double dj = fabs(Jnew[i] - Jold[i]);
        double e;
        if (dj == 0.0) e = 0.0;
        else if (Jnew[i] > 0.0) e = dj / Jnew[i];
        else e = INFINITY;
        if (e > r) r = e;
    }
    return r;
}

/*
 * Full solve (O3-O7). Outputs J, Gamma [N][G]; optionally every intensity I_out [D][N][G]
 * (final sweep). prev_init [D][N][G] seeds the periodic inflow (warm start) or NULL.
 * dc_n: 0 for transport scheme (a) of Sec. 2.6 (outflow split over the outflow faces by A n.Omega),
 * n > 0 for direction-conserving transport, scheme (b) (dc_choose: equal parts to the n faces most
 * nearly along Omega; the paper's n is the number of dimensions, 3).
 * law: OR_LAW_BALANCE (O3) or OR_LAW_EXP, the exponential reading of Sec. 2.6's "non-absorbed
 * inflow plus source": with tau = kappa_t V / P_c, the outgoing intensity is
 * (exp(-tau) F_in + q) / P_c and J is formed from the cell-mean intensity (F_in / P_c)(1 - exp(-tau))/tau,
 * so that kappa_t V times it is the removed flux; Gamma, the scattering source and the
 * conservation tally keep their form.
 * Returns OR_OK, OR_NOT_CONVERGED (outputs still written), or an error.
 */
int oracle_solve(int64_t n_cells, int64_t n_faces, const double* volume, const int32_t* face_cells,
                 const double* area, const double* normal, const uint8_t* flags, int32_t n_dir,
                 const double* omega, const double* weight, int32_t n_groups, const double* kappa_abs,
                 const double* kappa_scat, const double* emissivity, const double* bc_inflow, double tol_scat,
                 int32_t max_it_scat, double tol_pbc, int32_t max_it_pbc, const double* prev_init,
                 int fused, int law, int dc_n, int n_threads, double* J, double* Gam, double* I_out,
                 oracle_stats* st) {
    if (law != OR_LAW_BALANCE && law != OR_LAW_EXP) return OR_ERR_ARG;
    if (dc_n < 0) return OR_ERR_ARG;
    problem p;
    memset(&p, 0, sizeof p);
    p.n_cells = n_cells; p.n_faces = n_faces; p.volume = volume; p.face_cells = face_cells;
    p.area = area; p.normal = normal; p.flags = flags; p.n_dir = n_dir; p.omega = omega;
    p.weight = weight; p.n_groups = n_groups; p.kappa_abs = kappa_abs; p.kappa_scat = kappa_scat;
    p.emissivity = emissivity; p.bc_inflow = bc_inflow;
    memset(st, 0, sizeof *st);
    int rc = check_problem(&p);
    if (rc != OR_OK) return rc;
    rc = build_sides(&p);
    if (rc != OR_OK) { free_sides(&p); return rc; }
    int64_t N = n_cells, G = n_groups, NG = N * G, D = n_dir;
    int has_scat = 0, has_pbc = 0;
    if (kappa_scat)
        for (int64_t i = 0; i < NG; ++i)
            if (kappa_scat[i] != 0.0) { has_scat = 1; break; }
    for (int64_t f = 0; f < n_faces; ++f)
        if (flags[f] & OR_FACE_PERIODIC) { has_pbc = 1; break; }
    p.law = law;
    p.dc_n = dc_n;
    dc_scratch x;
    if (dc_scratch_init(&p, &x) != OR_OK) { dc_scratch_free(&x); free_sides(&p); return OR_ERR_MEM; }
    if (law == OR_LAW_EXP) {
        p.mean = (double*)calloc((size_t)(D * NG > 0 ? D * NG : 1), sizeof(double));
        if (!p.mean) { dc_scratch_free(&x); free_sides(&p); return OR_ERR_MEM; }
    }
    double* I = (double*)calloc((size_t)(D * NG > 0 ? D * NG : 1), sizeof(double));
    double* Iprev = (double*)calloc((size_t)(D * NG > 0 ? D * NG : 1), sizeof(double));
    double* q = (double*)malloc(sizeof(double) * (size_t)(NG > 0 ? NG : 1));
    double* Jold = (double*)calloc((size_t)(NG > 0 ? NG : 1), sizeof(double));
    double* jn = (double*)calloc((size_t)(NG > 0 ? NG : 1), sizeof(double));
    double* jn1 = (double*)calloc((size_t)(NG > 0 ? NG : 1), sizeof(double));
    if (!I || !Iprev || !q || !Jold || !jn || !jn1) { rc = OR_ERR_MEM; goto out; }
    if (has_pbc && prev_init) memcpy(Iprev, prev_init, sizeof(double) * (size_t)(D * NG));
    if (has_pbc) periodic_source(&p, Iprev, jn, &x);
    int conv_pbc = !has_pbc, conv_scat = !has_scat;
    int it_pbc = 0, it_scat_total = 0;
    double res_pbc = 0.0, res_pbc_mean = 0.0, res_scat = 0.0;
    if (fused && has_scat && has_pbc) {
        /* Both loops fused (the speed-up Sec. 2.7 proposes): every sweep takes the scattering source
         * from the latest J and the periodic inflow from the previous sweep; stop when both changes
         * are below their tolerances. J is not reset between periodic iterations. */
        for (;;) {
            for (int64_t c = 0; c < N; ++c)
                for (int g = 0; g < G; ++g) {
                    double ks = kappa_scat[c * G + g];
                    q[c * G + g] = emissivity[c * G + g] / FOURPI + ks * volume[c] * Jold[c * G + g];
                }
            rc = run_dirs(&p, n_threads, 0, q, 0, Iprev, I, NULL, NULL, 1);
            if (rc != OR_OK) goto out;
            ++it_scat_total;
            ++it_pbc;
            mean_intensity(&p, tally_field(&p, I), J);
            res_scat = scat_residual(NG, J, Jold);
            memcpy(Jold, J, sizeof(double) * (size_t)NG);
            periodic_source(&p, I, jn1, &x);
            double emax = 0.0, esum = 0.0;
            for (int64_t i = 0; i < NG; ++i) {
                double s = jn1[i] + jn[i];
                double e = s > 0.0 ? fabs(jn1[i] - jn[i]) / s : 0.0;
                if (e > emax) emax = e;
                esum += e;
            }
            res_pbc = emax;
            res_pbc_mean = NG > 0 ? esum / (double)NG : 0.0;
            memcpy(jn, jn1, sizeof(double) * (size_t)NG);
            memcpy(Iprev, I, sizeof(double) * (size_t)(D * NG));
            conv_pbc = res_pbc < tol_pbc;
            conv_scat = res_scat <= tol_scat;
            if (conv_pbc && conv_scat) break;
            if (it_pbc >= max_it_pbc) break;
        }
    }
    for (; !(fused && has_scat && has_pbc);) {
        /* O5: source iteration with the periodic inflow Iprev held fixed */
        for (int64_t i = 0; i < NG; ++i) Jold[i] = 0.0;
        int it_scat = 0;
        for (;;) {
            for (int64_t c = 0; c < N; ++c)
                for (int g = 0; g < G; ++g) {
                    double ks = kappa_scat ? kappa_scat[c * G + g] : 0.0;
                    q[c * G + g] = emissivity[c * G + g] / FOURPI + ks * volume[c] * Jold[c * G + g];
                }
            rc = run_dirs(&p, n_threads, 0, q, 0, has_pbc ? Iprev : NULL, I, NULL, NULL, 1);
            if (rc != OR_OK) goto out;
            ++it_scat;
            mean_intensity(&p, tally_field(&p, I), J);
            if (!has_scat) break;
            res_scat = scat_residual(NG, J, Jold);
            memcpy(Jold, J, sizeof(double) * (size_t)NG);
            if (res_scat <= tol_scat) { conv_scat = 1; break; }
            if (it_scat >= max_it_scat) { conv_scat = 0; break; }
        }
        it_scat_total += it_scat;
        ++it_pbc;
        if (!has_pbc) break;
        /* O6: sources for the next sweep and their relative change */
        periodic_source(&p, I, jn1, &x);
        double emax = 0.0, esum = 0.0;
        for (int64_t i = 0; i < NG; ++i) {
            double s = jn1[i] + jn[i];
            double e = s > 0.0 ? fabs(jn1[i] - jn[i]) / s : 0.0;
            if (e > emax) emax = e;
            esum += e;
        }
        res_pbc = emax;
        res_pbc_mean = NG > 0 ? esum / (double)NG : 0.0;
        memcpy(jn, jn1, sizeof(double) * (size_t)NG);
        memcpy(Iprev, I, sizeof(double) * (size_t)(D * NG));
        if (res_pbc < tol_pbc) { conv_pbc = 1; break; }
        if (it_pbc >= max_it_pbc) { conv_pbc = 0; break; }
    }
    tallies(&p, I, J, Gam, st, &x);
    st->it_scat = it_scat_total;
    st->it_pbc = it_pbc;
    st->res_scat = res_scat;
    st->res_pbc = res_pbc;
    st->res_pbc_mean = res_pbc_mean;
    if (I_out) memcpy(I_out, I, sizeof(double) * (size_t)(D * NG));
    rc = (conv_pbc && conv_scat) ? OR_OK : OR_NOT_CONVERGED;
out:
    free(I); free(Iprev); free(q); free(Jold); free(jn); free(jn1); free(p.mean);
    dc_scratch_free(&x);
    free_sides(&p);
    return rc;
}

/*
 * O9: adjoint of a loss L(J, Gamma), with or without isotropic scattering and periodic faces.
 * dl_dJ, dl_dGamma [N][G] (either may be NULL = 0). Outputs grad_kappa_abs, grad_emissivity
 * and, if not NULL, grad_kappa_scat [N][G].
 *
 * The forward state is oracle_solve's (the source iteration of Alg. 1 inside the periodic
 * iteration of Sec. 2.7, both to their tolerances). Write the converged system as A I = b with
 *   (A I)_d = L_d I_d - P_d I_d - kappa_s V J,   J = (1/4pi) sum_d w_d I_d,
 * L_d the transport operator without periodic faces and P_d the periodic inflow coupling. Its
 * transpose is solved for lambda with
 *   g_{d,c} = w_d (dl_dGamma_c kappa_a,c V_c + dl_dJ_c / 4pi)        (dL/dI_{c,d})
 *   L_d^T lambda_d = g_d + P_d^T lambda_d + w_d kappa_s,c V_c mu_c / 4pi,  mu_c = sum_d lambda_{d,c}
 * by one transposed iteration that lags both couplings by a pass: mu and the periodic lambda start
 * at 0; each pass sweeps every direction in reversed topological order, reading the partner's
 * lambda of the previous pass across each periodic outflow side (P_d^T), then recomputes mu. It
 * stops when max |mu_new - mu_old| <= tol_scat * max |mu_new| (0/0 counts as converged) or after
 * max_it_scat passes. Then
 *   dL/dkappa_a,c = sum_d V_c I_{c,d} (w_d dl_dGamma_c - lambda_{d,c})
 *   dL/deps_c     = sum_d lambda_{d,c} / 4pi
 *   dL/dkappa_s,c = sum_d V_c lambda_{d,c} (J_c - I_{c,d})
 * Without either coupling one transposed sweep gives lambda exactly. iters (or NULL) receives the
 * forward sweep count and the transposed pass count. Returns OR_NOT_CONVERGED (gradients still
 * written) when the forward solve or the transposed iteration hit its maximum.
 */
int oracle_adjoint(int64_t n_cells, int64_t n_faces, const double* volume, const int32_t* face_cells,
                   const double* area, const double* normal, const uint8_t* flags, int32_t n_dir,
                   const double* omega, const double* weight, int32_t n_groups, const double* kappa_abs,
                   const double* kappa_scat, const double* emissivity, const double* bc_inflow,
                   const double* dl_dJ, const double* dl_dGamma, double tol_scat, int32_t max_it_scat,
                   double tol_pbc, int32_t max_it_pbc, int n_threads, double* grad_kappa_abs,
                   double* grad_emissivity, double* grad_kappa_scat, int32_t* iters) {
    if (max_it_scat < 1 || max_it_pbc < 1) return OR_ERR_ARG;
    problem p;
    memset(&p, 0, sizeof p);
    p.n_cells = n_cells; p.n_faces = n_faces; p.volume = volume; p.face_cells = face_cells;
    p.area = area; p.normal = normal; p.flags = flags; p.n_dir = n_dir; p.omega = omega;
    p.weight = weight; p.n_groups = n_groups; p.kappa_abs = kappa_abs; p.kappa_scat = kappa_scat;
    p.emissivity = emissivity; p.bc_inflow = bc_inflow;
    int rc = check_problem(&p);
    if (rc != OR_OK) return rc;
    int64_t N = n_cells, G = n_groups, NG = N * G, D = n_dir;
    int has_scat = 0, has_pbc = 0;
    if (kappa_scat)
        for (int64_t i = 0; i < NG; ++i)
            if (kappa_scat[i] != 0.0) { has_scat = 1; break; }
    for (int64_t f = 0; f < n_faces; ++f)
        if (flags[f] & OR_FACE_PERIODIC) { has_pbc = 1; break; }
    double* I = (double*)calloc((size_t)(D * NG > 0 ? D * NG : 1), sizeof(double));
    double* J = (double*)calloc((size_t)(NG > 0 ? NG : 1), sizeof(double));
    double* Gam = (double*)calloc((size_t)(NG > 0 ? NG : 1), sizeof(double));
    double* lam = (double*)calloc((size_t)(D * NG > 0 ? D * NG : 1), sizeof(double));
    double* lam_prev = (double*)calloc((size_t)(D * NG > 0 ? D * NG : 1), sizeof(double));
    double* g = (double*)calloc((size_t)(D * NG > 0 ? D * NG : 1), sizeof(double));
    double* mu = (double*)calloc((size_t)(NG > 0 ? NG : 1), sizeof(double));
    int built = 0, conv_fwd = 1, conv_adj = 1, it_adj = 0;
    oracle_stats fst;
    if (!I || !J || !Gam || !lam || !lam_prev || !g || !mu) { rc = OR_ERR_MEM; goto out; }
    /* forward: the converged state, every intensity of the final sweep */
    rc = oracle_solve(n_cells, n_faces, volume, face_cells, area, normal, flags, n_dir, omega, weight, n_groups,
                      kappa_abs, kappa_scat, emissivity, bc_inflow, tol_scat, max_it_scat, tol_pbc, max_it_pbc,
                      NULL, 0, OR_LAW_BALANCE, 0, n_threads, J, Gam, I, &fst);
    if (rc == OR_NOT_CONVERGED) conv_fwd = 0;
    else if (rc != OR_OK) goto out;
    rc = build_sides(&p);
    built = 1;
    if (rc != OR_OK) goto out;
    /* the transposed iteration */
    for (;;) {
        for (int32_t d = 0; d < n_dir; ++d)
            for (int64_t c = 0; c < N; ++c)
                for (int k = 0; k < G; ++k) {
                    int64_t i = c * G + k;
                    double gd = dl_dGamma ? dl_dGamma[i] * kappa_abs[i] * volume[c] : 0.0;
                    double gj = dl_dJ ? dl_dJ[i] / FOURPI : 0.0;
                    double gs = has_scat ? kappa_scat[i] * volume[c] * mu[i] / FOURPI : 0.0;
                    g[(int64_t)d * NG + i] = weight[d] * (gd + gj + gs);
                }
        rc = run_dirs(&p, n_threads, 1, g, NG, has_pbc ? lam_prev : NULL, lam, NULL, NULL, 1);
        if (rc != OR_OK) goto out;
        ++it_adj;
        if (!has_scat && !has_pbc) break;
        double dmax = 0.0, mmax = 0.0;
        for (int64_t i = 0; i < NG; ++i) {
            double m = 0.0;
            for (int32_t d = 0; d < n_dir; ++d) m += lam[(int64_t)d * NG + i];
            double dm = fabs(m - mu[i]);
            if (dm > dmax) dmax = dm;
            if (fabs(m) > mmax) mmax = fabs(m);
            mu[i] = m;
        }
        if (has_pbc) memcpy(lam_prev, lam, sizeof(double) * (size_t)(D * NG));
        if (dmax == 0.0 || dmax <= tol_scat * mmax) break;
        if (it_adj >= max_it_scat) { conv_adj = 0; break; }
    }
    for (int64_t c = 0; c < N; ++c)
        for (int k = 0; k < G; ++k) {
            int64_t i = c * G + k;
            double gk = 0.0, ge = 0.0, gs = 0.0;
            double rg = dl_dGamma ? dl_dGamma[i] : 0.0;
            for (int32_t d = 0; d < n_dir; ++d) {
                double Icd = I[(int64_t)d * NG + i];
                double lcd = lam[(int64_t)d * NG + i];
                gk += volume[c] * Icd * (weight[d] * rg - lcd);
                ge += lcd / FOURPI;
                gs += volume[c] * lcd * (J[i] - Icd);
            }
            grad_kappa_abs[i] = gk;
            grad_emissivity[i] = ge;
            if (grad_kappa_scat) grad_kappa_scat[i] = gs;
        }
    if (iters) { iters[0] = fst.it_scat; iters[1] = it_adj; }
    rc = (conv_fwd && conv_adj) ? OR_OK : OR_NOT_CONVERGED;
out:
    free(I); free(J); free(Gam); free(lam); free(lam_prev); free(g); free(mu);
    if (built) free_sides(&p);
    return rc;
}

/* ------------------------------------------------------------------------------------------------
 * Remap coefficients between two direction sets (Sec. 2.6, the rotation paragraph): after the
 * directions are rotated, an angle-dependent quantity is carried over as
 *   I(Omega'_i) = sum_j c_ij I(Omega_j),  c_ij = dS_ij / dS_i,
 * dS_ij the solid angle that the bin of the new direction i shares with the bin of the old direction
 * j, dS_i = sum_j dS_ij the solid angle of bin i (so every row sums to 1). A direction's bin is the part
 * of the unit sphere nearer to it than to any other direction of its set. The solid angles are taken
 * by quadrature: n_quad points of a Fibonacci sphere,
 *   z_m = 1 - (2m + 1)/n_quad,  phi_m = m pi (3 - sqrt 5),
 * each of equal weight, each in the bin of the direction with the largest p.Omega
 * (((px Ox) + (py Oy)) + (pz Oz), separately rounded; ties to the lower index); dS_ij is then
 * proportional to the number of points in both bin i and bin j.
 * c_out[n_dir][n_dir] row-major, row i = new direction i.
 * ------------------------------------------------------------------------------------------------ */
static int32_t nearest_direction(const double* p, int32_t n_dir, const double* omega) {
    int32_t best = 0;
    double bd = -2.0;
    for (int32_t d = 0; d < n_dir; ++d) {
        double t = ((p[0] * omega[3 * d]) + (p[1] * omega[3 * d + 1])) + (p[2] * omega[3 * d + 2]);
        if (t > bd) {
            bd = t;
            best = d;
        }
    }
    return best;
}

int oracle_remap_coeffs(int32_t n_dir, const double* omega_old, const double* omega_new, int64_t n_quad,
                        double* c_out) {
    if (n_dir < 1 || n_quad < 1 || !omega_old || !omega_new || !c_out) return OR_ERR_ARG;
    int64_t* cnt = (int64_t*)calloc((size_t)n_dir * (size_t)n_dir, sizeof(int64_t));
    int64_t* row = (int64_t*)calloc((size_t)n_dir, sizeof(int64_t));
    if (!cnt || !row) {
        free(cnt);
        free(row);
        return OR_ERR_MEM;
    }
    const double golden = M_PI * (3.0 - sqrt(5.0));
    for (int64_t m = 0; m < n_quad; ++m) {
        double z = 1.0 - (2.0 * (double)m + 1.0) / (double)n_quad;
        double r = sqrt(1.0 - z * z);
        double ph = (double)m * golden;
        double p[3] = {r * cos(ph), r * sin(ph), z};
        int32_t i = nearest_direction(p, n_dir, omega_new);
        int32_t j = nearest_direction(p, n_dir, omega_old);
        cnt[(int64_t)i * n_dir + j]++;
        row[i]++;
    }
    for (int32_t i = 0; i < n_dir; ++i)
        for (int32_t j = 0; j < n_dir; ++j)
            c_out[(int64_t)i * n_dir + j] = row[i] > 0 ? (double)cnt[(int64_t)i * n_dir + j] / (double)row[i] : 0.0;
    free(cnt);
    free(row);
    return OR_OK;
}
