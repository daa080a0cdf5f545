// Host side of the C ABI declared in include/sweep.h: context, uploads and validation,
// the solve loop (periodic iteration of Sec. 2.7 outside, source iteration of Alg. 1 inside,
// batched sweep innermost), the schedule autotuner and the adjoint with recompute batches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "adjoint.cuh"
#include "common.cuh"

using namespace sw;


struct SolveBuf {
    void* I[2] = {nullptr, nullptr};
    int sign[2] = {0, 0};   // sign bit currently carried by every value of the buffer
    size_t bytes = 0;
    int prec = 0;
    int last = -1;          // buffer holding the last solve's final intensities
    int64_t N = 0;
    int nd = 0, G = 0;
};

struct sweep_ctx {
    int device = 0;
    cudaStream_t st = nullptr;
    int sms = 0;
    std::string err;
    // mesh
    bool has_mesh = false;
    DevMesh mesh;
    // directions
    bool has_dirs = false;
    int D = 0;
    double* om64 = nullptr;
    double* w64 = nullptr;
    float4* om32 = nullptr;
    float4* om32lo = nullptr;  // [D] direction minus its FP32 value
    double wsum = 0.0;
    // material
    bool has_mat = false;
    int G = 0;
    double *ka = nullptr, *ks = nullptr, *em = nullptr, *bc = nullptr;
    bool has_scat = false;
    // forward levels (all directions) and adjoint batch levels
    Levels lev, adj_lev;
    // solution
    SolveBuf sb;
    float2* cm32 = nullptr;
    double2* cm64 = nullptr;
    size_t cm_cap = 0;  // elements
    double *J = nullptr, *Jold = nullptr, *Gam = nullptr, *jn = nullptr, *jn1 = nullptr;
    size_t ng_cap = 0;
    double* partial = nullptr;
    int partial_cap = 0;
    int last_kernel = SWEEP_KERNEL_NONE;  // form of the last batched sweep launched
    double* red = nullptr;          // [4]
    unsigned long long* dmax = nullptr;
    GridBar* bar = nullptr;
    int* derr = nullptr;
    int64_t* scratch = nullptr;
    float* stall_word = nullptr;
    // adjoint buffers
    void* adjI = nullptr;
    void* adjL = nullptr;
    size_t adj_bytes_I = 0, adj_bytes_L = 0;
    // the boundary inflow in FP32 for the FP32 sweeps, converted once per material
    float* bc32 = nullptr;
    bool bc32_ready = false;
    // EXP law: cell-mean intensities of the last sweep, [nd][N][G] in the solve precision
    void* Imean = nullptr;
    size_t imean_bytes = 0;
    // autotuner: schedule and block size per (precision, G)
    int tuned[2][9][3][4] = {};  // [precision][groups][operator form OPF_*] -> schedule, threads, lanes, blocks/SM
    int64_t launches = 0;  // kernels launched by this context
    PeriodicTable ptab;          // periodic-inflow weights, rebuilt at the start of each periodic solve
    cudaStream_t gst = nullptr;  // capture/replay stream of the iteration graphs
    void* hpin = nullptr;        // pinned host words the iteration graphs write
};

namespace {

sweep_status cuda_status(sweep_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return SWEEP_OK;
    c->err = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SWEEP_ERR_OOM : SWEEP_ERR_CUDA;
}

#define CK(x, what)                                       \
    do {                                                  \
        cudaError_t _e = (x);                             \
        if (_e != cudaSuccess) return cuda_status(c, _e, what); \
    } while (0)
// a checked call that launches one kernel
#define CKL(x, what)     \
    do {                 \
        ++c->launches;   \
        CK(x, what);     \
    } while (0)

sweep_status bad(sweep_ctx* c, const std::string& m) {
    c->err = m;
    return SWEEP_ERR_INVALID_ARG;
}

template <typename T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

void free_levels(Levels& L) {
    dfree(L.raw); dfree(L.task); dfree(L.trec); dfree(L.info); dfree(L.level); dfree(L.lvl_cnt); dfree(L.pad_off);
    dfree(L.lev_chunk); dfree(L.seg_off); dfree(L.op); dfree(L.dlev);
    for (PackedOp* P : {&L.pk, &L.pkt}) {
        dfree(P->pk); dfree(P->meta); dfree(P->lev_pk); dfree(P->grp); dfree(P->lev_grp); dfree(P->cnt);
        dfree(P->off); dfree(P->scan); dfree(P->flag);
    }
    dfree(L.lfill);
    dfree(L.dc_mask); dfree(L.dc_inm); dfree(L.dc_share32); dfree(L.dc_share64);
    L = Levels();
}

void free_mesh(DevMesh& m) {
    dfree(m.rowptr); dfree(m.side); dfree(m.side64); dfree(m.side_lo); dfree(m.nbr_rows); dfree(m.twin); dfree(m.vol);
    dfree(m.pcells); dfree(m.bcells);
    m = DevMesh();
}

void free_solution(sweep_ctx* c) {
    dfree(c->sb.I[0]); dfree(c->sb.I[1]);
    c->sb = SolveBuf();
    dfree(c->adjI); dfree(c->adjL);
    c->adj_bytes_I = c->adj_bytes_L = 0;
    dfree(c->Imean);
    c->imean_bytes = 0;
}

void free_material(sweep_ctx* c) {
    dfree(c->ka); dfree(c->ks); dfree(c->em); dfree(c->bc); dfree(c->bc32);
    c->bc32_ready = false;
    c->has_mat = false;
    c->has_scat = false;
}

int dir_bits(int nd) {
    int b = 1;
    while ((1 << b) < nd) ++b;
    return b;
}

sweep_status alloc_levels(sweep_ctx* c, Levels& L, int d0, int nd) {
    const int64_t N = c->mesh.N;
    if (L.nd == nd && L.raw && L.d0 == d0) {
        L.valid = false;
        L.op_valid = false;
        L.pkt.valid = false;
        return SWEEP_OK;
    }
    free_levels(L);
    L.d0 = d0;
    L.nd = nd;
    int bits = dir_bits(nd);
    L.cshift = 32 - bits;
    L.cmask = (bits == 32) ? 0u : ((1u << L.cshift) - 1u);
    if ((uint64_t)N > (uint64_t)L.cmask + 1ull) return bad(c, "n_cells too large for the number of directions");
    L.task_cap = N * (int64_t)nd + 32 * (N + 2);
    CK(cudaMalloc(&L.raw, sizeof(uint32_t) * L.task_cap), "alloc task list");
    CK(cudaMalloc(&L.task, sizeof(uint32_t) * L.task_cap), "alloc task list");
    CK(cudaMalloc(&L.trec, sizeof(int4) * L.task_cap), "alloc task records");
    CK(cudaMalloc(&L.info, sizeof(int4) * N * nd), "alloc classification");
    CK(cudaMalloc(&L.level, sizeof(int32_t) * N * nd), "alloc levels");
    CK(cudaMalloc(&L.lvl_cnt, sizeof(int32_t) * (N + 2)), "alloc level counts");
    CK(cudaMalloc(&L.pad_off, sizeof(uint32_t) * (N + 2)), "alloc level offsets");
    CK(cudaMalloc(&L.lev_chunk, sizeof(int64_t) * (N + 2)), "alloc level chunks");
    L.dlev_cap = (int)std::min<int64_t>(N + 1, 1 << 16);
    CK(cudaMalloc(&L.dlev, sizeof(int32_t) * ((int64_t)nd * (2 * L.dlev_cap + 2) + 1)), "alloc level tables");
    // worst case of levels x (nd+1) segment starts is only known after levelisation
    return SWEEP_OK;
}

sweep_status run_levelise(sweep_ctx* c, Levels& L, int d0, int nd, long long budget, float* t1, float* t2,
                          int transport = 0) {
    sweep_status s = alloc_levels(c, L, d0, nd);
    if (s != SWEEP_OK) return s;
    // scheme (b) tables, [N][nd] each (freed when scheme (a) is levelised again)
    if (transport > 0 && !L.dc_mask) {
        const size_t n = (size_t)c->mesh.N * nd;
        CK(cudaMalloc(&L.dc_mask, sizeof(uint64_t) * n), "alloc scheme (b) tables");
        CK(cudaMalloc(&L.dc_inm, sizeof(uint64_t) * n), "alloc scheme (b) tables");
        CK(cudaMalloc(&L.dc_share32, sizeof(float) * n), "alloc scheme (b) tables");
        CK(cudaMalloc(&L.dc_share64, sizeof(double) * n), "alloc scheme (b) tables");
    } else if (transport == 0 && L.dc_mask) {
        dfree(L.dc_mask); dfree(L.dc_inm); dfree(L.dc_share32); dfree(L.dc_share64);
    }
    L.transport = transport;
    CK(cudaMemsetAsync(c->derr, 0, sizeof(int), c->st), "reset error word");
    std::string msg;
    CK(levelise(c->mesh, L, c->om64, c->om32, c->om32lo, c->sms, c->bar, c->derr, budget, c->scratch, c->st, t1, t2, &msg),
       "levelise");
    c->launches += 3;  // classification, levelisation, per-level direction grouping
    if (!L.valid) {
        c->err = msg;
        if (msg.find("cyclic") != std::string::npos) return SWEEP_ERR_CYCLE;
        if (msg.find("direction-conserving") != std::string::npos) return SWEEP_ERR_INVALID_ARG;
        return SWEEP_ERR_TIMEOUT;
    }
    return SWEEP_OK;
}

long long budget_of(const sweep_opts* o) { return o && o->spin_budget > 0 ? o->spin_budget : (1ll << 21); }

sweep_status ensure_common(sweep_ctx* c) {
    if (!c->bar) {
        CK(cudaMalloc(&c->bar, sizeof(GridBar)), "alloc");
        CK(cudaMalloc(&c->derr, sizeof(int)), "alloc");
        CK(cudaMalloc(&c->scratch, sizeof(int64_t) * 4), "alloc");
        CK(cudaMalloc(&c->red, sizeof(double) * 4), "alloc");
        CK(cudaMalloc(&c->dmax, 2 * sizeof(unsigned long long)), "alloc");  // [0] periodic or scattering, [1] scattering when fused
        CK(cudaMalloc(&c->stall_word, sizeof(double)), "alloc");
        CK(cudaMemset(c->stall_word, 0, sizeof(double)), "init");
    }
    return SWEEP_OK;
}

sweep_status ensure_ng(sweep_ctx* c, size_t ng) {
    if (c->ng_cap >= ng && c->J) return SWEEP_OK;
    dfree(c->J); dfree(c->Jold); dfree(c->Gam); dfree(c->jn); dfree(c->jn1);
    size_t n = ng > 0 ? ng : 1;
    CK(cudaMalloc(&c->J, sizeof(double) * n), "alloc J");
    CK(cudaMalloc(&c->Jold, sizeof(double) * n), "alloc J");
    CK(cudaMalloc(&c->Gam, sizeof(double) * n), "alloc Gamma");
    CK(cudaMalloc(&c->jn, sizeof(double) * n), "alloc j");
    CK(cudaMalloc(&c->jn1, sizeof(double) * n), "alloc j");
    c->ng_cap = n;
    return SWEEP_OK;
}

sweep_status ensure_cm(sweep_ctx* c, size_t n) {
    if (c->cm_cap >= n && c->cm32) return SWEEP_OK;
    dfree(c->cm32); dfree(c->cm64);
    size_t m = n > 0 ? n : 1;
    CK(cudaMalloc(&c->cm32, sizeof(float2) * m), "alloc sources");
    CK(cudaMalloc(&c->cm64, sizeof(double2) * m), "alloc sources");
    c->cm_cap = m;
    return SWEEP_OK;
}

sweep_status ensure_partial(sweep_ctx* c, int nblk) {
    if (c->partial_cap >= nblk && c->partial) return SWEEP_OK;
    dfree(c->partial);
    CK(cudaMalloc(&c->partial, sizeof(double) * 2 * (nblk > 0 ? nblk : 1)), "alloc partials");
    c->partial_cap = nblk;
    return SWEEP_OK;
}

int nblocks256(int64_t n) { return (int)((n + 255) / 256 > 0 ? (n + 255) / 256 : 1); }

// A timing event that is destroyed when it goes out of scope, also on the error returns. Destroying an
// event that the device has not reached yet is allowed: its resources are freed once it completes.
struct ScopedEvent {
    cudaEvent_t e = nullptr;
    ScopedEvent() { cudaEventCreate(&e); }
    ~ScopedEvent() {
        if (e) cudaEventDestroy(e);
    }
    ScopedEvent(const ScopedEvent&) = delete;
    ScopedEvent& operator=(const ScopedEvent&) = delete;
    operator cudaEvent_t() const { return e; }
};

// cell update of the packed kernel for these arguments
int pk_mode(const SweepArgs& a) { return a.reverse ? PK_TRANSPOSED : (a.law ? PK_EXP : PK_BALANCE); }

SweepArgs make_args(sweep_ctx* c, const Levels& L, int precision, const void* cm, void* I, const void* Iprev,
                    int G, int parity, int reverse, int level_sync, const sweep_opts* o) {
    SweepArgs a;
    memset(&a, 0, sizeof a);
    a.task = L.task;
    a.trec = L.trec;
    // the EXP law runs in the packed, generic and plain kernels; the adjoint takes BALANCE
    a.law = (!reverse && o) ? o->law : SWEEP_LAW_BALANCE;
    a.Imean = a.law ? c->Imean : nullptr;
    const bool opr = precision == 32 && !(o && o->geometry_only);
    // forward: the assembled operator of the levels; transposed: the packed transposed operator
    const PackedOp* P = nullptr;
    if (opr && !reverse && L.op_valid && L.op_format == OPF_PACKETS) P = &L.pk;
    if (opr && reverse && L.pkt.valid) P = &L.pkt;
    a.op = opr && !reverse && !a.law && L.op_valid && L.op_format == OPF_LINES ? L.op : nullptr;
    if (P) {
        a.pk = P->pk;
        a.pk_meta = P->meta;
        a.n_pk = P->n_pk;
        a.lev_pk = P->lev_pk;
    }
    if (L.transport > 0 && !reverse) {
        a.dc_mask = L.dc_mask;
        a.dc_share32 = L.dc_share32;
        a.dc_share64 = L.dc_share64;
        a.twin = c->mesh.twin;
    }
    a.n_chunks = L.h_lev_chunk.empty() ? 0 : L.h_lev_chunk.back();
    a.lev_chunk = L.lev_chunk;
    a.n_levels = L.n_levels;
    a.cshift = L.cshift;
    a.cmask = L.cmask;
    a.nd = L.nd;
    a.rowptr = c->mesh.rowptr;
    a.side = c->mesh.side;
    a.side64 = c->mesh.side64;
    a.side_lo = c->mesh.side_lo;
    a.om32 = c->om32 + L.d0;
    a.om32lo = c->om32lo + L.d0;
    a.om64 = c->om64 + 3 * (int64_t)L.d0;
    a.w64 = c->w64 + L.d0;
    a.cm = cm;
    a.bc = reverse ? nullptr : (precision == 64 ? (const void*)c->bc : nullptr);
    a.I = I;
    a.Iprev = Iprev;
    a.N = c->mesh.N;
    a.G = G;
    a.parity = parity;
    a.reverse = reverse;
    a.level_sync = level_sync;
    a.bar = c->bar;
    a.err = c->derr;
    a.spin_budget = budget_of(o);
    a.debug_stall = o ? o->debug_stall : 0;
    a.stall_word = c->stall_word;
    (void)precision;
    return a;
}

sweep_status run_sweep(sweep_ctx* c, const Levels& L, int precision, int schedule, int threads, int lanes, int bpsm,
                       SweepArgs a, const float* bc32, float* ms) {
    if (precision == 32) a.bc = a.reverse ? nullptr : bc32;
    a.lanes = lanes;
    ScopedEvent e0, e1;
    CK(cudaMemsetAsync(c->bar, 0, sizeof(GridBar), c->st), "reset barrier");
    CK(cudaMemsetAsync(c->derr, 0, sizeof(int), c->st), "reset error word");
    cudaEventRecord(e0, c->st);
    if (schedule == SWEEP_SCHED_PLAIN) {
        c->last_kernel = SWEEP_KERNEL_PLAIN;
        const int nd = L.nd;
        for (int d = 0; d < nd; ++d) {
            for (int li = 0; li < L.n_levels; ++li) {
                const int lv = a.reverse ? L.n_levels - 1 - li : li;
                uint32_t b0 = L.h_seg_off[(size_t)lv * (nd + 1) + d], b1 = L.h_seg_off[(size_t)lv * (nd + 1) + d + 1];
                if (b1 > b0) CKL(launch_plain_level(a, b0, b1, c->st), "plain sweep");
            }
        }
    } else {
        const int fmt = a.pk ? OPF_PACKETS : (a.op ? OPF_LINES : OPF_NONE);
        // without an assembled operator the adjoint, the EXP law and scheme (b) run in the generic kernel
        const bool generic = fmt == OPF_NONE && (a.reverse || a.law || a.dc_mask);
        int per_sm = sweep_occupancy(precision, a.G, threads, L.nd, lanes, generic, fmt, pk_mode(a));
        if (per_sm < 1) return bad(c, "sweep kernel does not fit on an SM");
        if (bpsm > 0 && bpsm < per_sm) per_sm = bpsm;
        a.level_sync = schedule == SWEEP_SCHED_LEVEL ? 1 : 0;
        CKL(launch_sweep(a, precision, c->sms * per_sm, threads, c->st, &c->last_kernel), "sweep launch");
    }
    cudaEventRecord(e1, c->st);
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, c->derr, sizeof herr, cudaMemcpyDeviceToHost, c->st), "read error word");
    CK(cudaStreamSynchronize(c->st), "sweep");
    float t = 0;
    cudaEventElapsedTime(&t, e0, e1);
    if (ms) *ms += t;
    if (herr != DEV_OK) {
        c->err = "sweep: a bounded device wait gave up";
        return SWEEP_ERR_TIMEOUT;
    }
    return SWEEP_OK;
}

// ---------------------------------------------------------------------------------------------
// The periodic iteration (Sec. 2.7) or the source iteration (Alg. 1) as CUDA graphs. The iterations
// of a solve repeat with a short period: which intensity buffer is swept, the sign parity it is
// written with, and which periodic-inflow array is read change in a cycle of 4 (periodic) or 2
// (scattering). Each distinct iteration is captured once per solve on the context's capture stream
// and replayed; an iteration is then one graph launch and one synchronisation, after which the
// host reads the convergence residual, the error word and the sweep's event times from pinned
// memory written by the graph itself.
// ---------------------------------------------------------------------------------------------
struct IterHost {
    int err;
    int pad;
    unsigned long long dmax;
    double red[2];
    unsigned long long dmax_scat;  // scattering change of a fused iteration
};

struct GraphSet {
    cudaGraphExec_t ex[4] = {};
    cudaEvent_t ev[4][3] = {};
    ~GraphSet() {
        for (int t = 0; t < 4; ++t) {
            if (ex[t]) cudaGraphExecDestroy(ex[t]);
            for (auto& e : ev[t])
                if (e) cudaEventDestroy(e);
        }
    }
};

// Captures whatever `enqueue` issues on stream gs into an executable graph; false (nothing run) if
// capture or instantiation is refused.
template <typename Fn>
bool capture(cudaStream_t gs, Fn enqueue, cudaGraphExec_t* ex) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const cudaError_t e1 = enqueue();
    const cudaError_t e2 = cudaStreamEndCapture(gs, &g);
    if (e1 != cudaSuccess || e2 != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return false;
    }
    const cudaError_t e3 = cudaGraphInstantiate(ex, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) {
        cudaGetLastError();
        *ex = nullptr;
        return false;
    }
    return true;
}

sweep_status ensure_graph_stream(sweep_ctx* c) {
    if (!c->gst) CK(cudaStreamCreateWithFlags(&c->gst, cudaStreamNonBlocking), "create capture stream");
    if (!c->hpin) CK(cudaHostAlloc(&c->hpin, sizeof(IterHost), cudaHostAllocDefault), "alloc pinned");
    return SWEEP_OK;
}

struct LoopState {
    int cur = 0, prev = -1;
    int it_pbc = 0, it_scat_total = 0, n_sweeps = 0;
    bool conv_pbc = false, conv_scat = false;
    double res_pbc = 0.0, res_pbc_mean = 0.0, res_scat = 0.0;
    float t_sweep = 0.f, t_other = 0.f;
};

// Runs the iterations of a solve as graphs: with exactly one of the two loops (periodic without
// scattering, or scattering without periodic faces), or with both fused (one source-iteration sweep per
// periodic iteration). *done = false (nothing run) when the graphs cannot be captured; the caller then
// runs the host loop from the same state.
sweep_status graph_loop(sweep_ctx* c, const sweep_opts& o, int prec, const void* cm, const float* bc32, int sched,
                        int threads, int lanes, int bpsm, int nblk, LoopState& st, bool* done) {
    *done = false;
    const bool pbc = c->mesh.n_pcells > 0;
    const bool scat = c->has_scat;
    const bool fused = pbc && scat;
    if (fused && !o.fused_loops) return SWEEP_OK;  // nested loops stay on the host
    SolveBuf& b = c->sb;
    const int64_t N = c->mesh.N;
    const int G = c->G, D = c->D;
    const size_t NG = (size_t)N * G;
    sweep_status s = ensure_graph_stream(c);
    if (s != SWEEP_OK) return s;
    cudaStream_t gs = c->gst;
    IterHost* hp = reinterpret_cast<IterHost*>(c->hpin);
    int fmt = (prec == 32 && c->lev.op_valid && !o.geometry_only) ? c->lev.op_format : OPF_NONE;
    if (o.law && fmt == OPF_LINES) fmt = OPF_NONE;  // the EXP law: packets or the mesh rows
    const bool generic = fmt == OPF_NONE && (o.law || c->lev.transport > 0);
    int per_sm = sweep_occupancy(prec, G, threads, c->lev.nd, lanes, generic ? 1 : 0, fmt,
                                 o.law ? PK_EXP : PK_BALANCE);
    if (per_sm < 1) return bad(c, "sweep kernel does not fit on an SM");
    if (bpsm > 0 && bpsm < per_sm) per_sm = bpsm;
    const int period = pbc ? 4 : 2;
    const int cur0 = st.cur;
    const int sgn[2] = {b.sign[0], b.sign[1]};
    double* jA = c->jn;
    double* jB = c->jn1;
    int kid = 0;
    // iteration type t: buffer, parity (the buffer's (t/2)-th or t-th write since the start), j arrays
    auto cur_of = [&](int t) { return pbc ? ((t & 1) ? 1 - cur0 : cur0) : cur0; };
    auto parity_of = [&](int t) {
        const int k = pbc ? t / 2 : t;  // writes of this buffer before iteration t, modulo 2
        return (k & 1) ? sgn[cur_of(t)] : !sgn[cur_of(t)];
    };
    auto enqueue = [&](int t, cudaEvent_t* ev) -> cudaError_t {
        cudaError_t e;
        const int cur = cur_of(t);
        if (scat) {  // scattering source from the previous J (Alg. 1)
            if ((e = launch_prep_material(N, G, c->mesh.vol, c->ka, c->ks, c->em, c->Jold,
                                          prec == 32 ? c->cm32 : nullptr, prec == 64 ? c->cm64 : nullptr, gs)))
                return e;
        }
        if ((e = cudaMemsetAsync(c->bar, 0, sizeof(GridBar), gs))) return e;
        if ((e = cudaMemsetAsync(c->derr, 0, sizeof(int), gs))) return e;
        if ((e = cudaEventRecordWithFlags(ev[0], gs, cudaEventRecordExternal))) return e;
        SweepArgs a = make_args(c, c->lev, prec, cm, b.I[cur], pbc ? b.I[1 - cur] : nullptr, G, parity_of(t), 0,
                                sched == SWEEP_SCHED_LEVEL ? 1 : 0, &o);
        a.debug_stall = 0;
        if (prec == 32) a.bc = bc32;
        a.lanes = lanes;
        if ((e = launch_sweep(a, prec, c->sms * per_sm, threads, gs, &kid))) return e;
        if ((e = cudaEventRecordWithFlags(ev[1], gs, cudaEventRecordExternal))) return e;
        if (scat) {
            if ((e = launch_tally(prec, o.law ? c->Imean : b.I[cur], N, G, D, 0, c->w64, c->wsum, c->mesh.vol, c->ka,
                                  c->em, c->J,
                                  c->Gam, c->partial, nblk, gs)))
                return e;
            unsigned long long* ds = c->dmax + (fused ? 1 : 0);
            if ((e = cudaMemsetAsync(ds, 0, sizeof(unsigned long long), gs))) return e;
            if ((e = launch_scat_residual(NG, c->J, c->Jold, ds, gs))) return e;
            if (fused && (e = cudaMemcpyAsync(&hp->dmax_scat, ds, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                              gs)))
                return e;
        }
        if (pbc) {
            double* jr = (t & 1) ? jB : jA;  // j of the previous iteration
            double* jw = (t & 1) ? jA : jB;
            if ((e = cudaMemsetAsync(c->dmax, 0, sizeof(unsigned long long), gs))) return e;
            if ((e = launch_periodic_source(prec, c->mesh, b.I[cur], G, D, c->om64, c->w64, jw, jr, c->dmax,
                                            c->partial, nblk, gs, &c->ptab)))
                return e;
            if ((e = launch_reduce_sum(c->partial, (int)c->mesh.n_pcells, c->red + 2, gs))) return e;
            if ((e = cudaMemcpyAsync(hp->red, c->red + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, gs))) return e;
        }
        if ((e = cudaEventRecordWithFlags(ev[2], gs, cudaEventRecordExternal))) return e;
        if ((e = cudaMemcpyAsync(&hp->err, c->derr, sizeof(int), cudaMemcpyDeviceToHost, gs))) return e;
        return cudaMemcpyAsync(&hp->dmax, c->dmax, sizeof(unsigned long long), cudaMemcpyDeviceToHost, gs);
    };
    const int max_it = pbc ? o.max_it_pbc : o.max_it_scat;
    const int ntypes = std::min(period, std::max(max_it, 1));
    GraphSet gset;
    for (int t = 0; t < ntypes; ++t) {
        for (auto& e : gset.ev[t]) CK(cudaEventCreate(&e), "create event");
        if (!capture(gs, [&] { return enqueue(t, gset.ev[t]); }, &gset.ex[t])) return SWEEP_OK;  // host loop instead
    }
    // the graphs run on the capture stream, after everything queued so far on the context's stream
    cudaEvent_t fork;
    CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming), "create event");
    cudaEventRecord(fork, c->st);
    cudaStreamWaitEvent(gs, fork, 0);
    cudaEventDestroy(fork);
    *done = true;
    const int per_iter = (pbc ? 3 : 1) + (scat ? 3 : 0);  // kernels per iteration
    for (int it = 0;; ++it) {
        const int t = it % period;
        CK(cudaGraphLaunch(gset.ex[t], gs), "graph launch");
        CK(cudaStreamSynchronize(gs), "iteration");
        c->launches += per_iter;
        c->last_kernel = kid;
        float ts = 0, to = 0;
        cudaEventElapsedTime(&ts, gset.ev[t][0], gset.ev[t][1]);
        cudaEventElapsedTime(&to, gset.ev[t][1], gset.ev[t][2]);
        st.t_sweep += ts;
        st.t_other += to;
        if (hp->err != DEV_OK) {
            c->err = "sweep: a bounded device wait gave up";
            return SWEEP_ERR_TIMEOUT;
        }
        const int cur = cur_of(t);
        b.sign[cur] = parity_of(t);
        ++st.n_sweeps;
        double r;
        memcpy(&r, &hp->dmax, sizeof r);
        if (pbc) {
            ++st.it_scat_total;
            ++st.it_pbc;
            st.res_pbc = r;
            st.res_pbc_mean = NG > 0 ? hp->red[0] / (double)NG : 0.0;
            std::swap(c->jn, c->jn1);
            st.prev = cur;
            st.cur = 1 - cur;
            if (fused) {
                memcpy(&st.res_scat, &hp->dmax_scat, sizeof st.res_scat);
                st.conv_pbc = st.res_pbc < o.tol_pbc;
                st.conv_scat = st.res_scat <= o.tol_scat;
                if (st.conv_pbc && st.conv_scat) break;
                if (st.it_pbc >= o.max_it_pbc) break;
                continue;
            }
            if (st.res_pbc < o.tol_pbc) { st.conv_pbc = true; break; }
            if (st.it_pbc >= o.max_it_pbc) { st.conv_pbc = false; break; }
        } else {
            ++st.it_scat_total;
            st.res_scat = r;
            if (st.res_scat <= o.tol_scat) { st.conv_scat = true; break; }
            if (st.it_scat_total >= o.max_it_scat) { st.conv_scat = false; break; }
        }
    }
    if (!pbc) st.it_pbc = 1;
    return SWEEP_OK;
}


}  // namespace

// ---------------------------------------------------------------------------------------------
extern "C" {

void sweep_default_opts(sweep_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->precision = 32;
    o->law = SWEEP_LAW_BALANCE;
    o->schedule = SWEEP_SCHED_AUTO;
    o->max_it_scat = 100;
    o->tol_scat = 1e-6;
    o->max_it_pbc = 100;
    o->tol_pbc = 1e-6;
    o->use_graph = 1;
}

const char* sweep_status_string(sweep_status s) {
    switch (s) {
        case SWEEP_OK: return "ok";
        case SWEEP_ERR_INVALID_ARG: return "invalid argument";
        case SWEEP_ERR_CYCLE: return "dependency graph is cyclic";
        case SWEEP_NOT_CONVERGED: return "iteration did not converge";
        case SWEEP_ERR_TIMEOUT: return "device wait timed out";
        case SWEEP_ERR_OOM: return "out of device memory";
        case SWEEP_ERR_CUDA: return "CUDA error";
    }
    return "unknown status";
}

const char* sweep_last_error(const sweep_ctx* c) { return c ? c->err.c_str() : "null context"; }

sweep_status sweep_create(sweep_ctx** out, int device, void* stream) {
    if (!out) return SWEEP_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return SWEEP_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) return SWEEP_ERR_CUDA;
    sweep_ctx* c = new sweep_ctx();
    c->device = device;
    c->st = (cudaStream_t)stream;
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
    if (!coop) {
        delete c;
        return SWEEP_ERR_CUDA;
    }
    sweep_status s = ensure_common(c);
    if (s != SWEEP_OK) {
        delete c;
        return s;
    }
    *out = c;
    return SWEEP_OK;
}

sweep_status sweep_destroy(sweep_ctx* c) {
    if (!c) return SWEEP_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->st);
    free_levels(c->lev);
    free_levels(c->adj_lev);
    free_solution(c);
    free_material(c);
    free_mesh(c->mesh);
    dfree(c->om64); dfree(c->w64); dfree(c->om32); dfree(c->om32lo);
    dfree(c->cm32); dfree(c->cm64);
    dfree(c->J); dfree(c->Jold); dfree(c->Gam); dfree(c->jn); dfree(c->jn1);
    dfree(c->partial); dfree(c->red); dfree(c->dmax); dfree(c->bar); dfree(c->derr); dfree(c->scratch);
    dfree(c->stall_word);
    dfree(c->ptab.off); dfree(c->ptab.wa);
    if (c->gst) cudaStreamDestroy(c->gst);
    if (c->hpin) cudaFreeHost(c->hpin);
    delete c;
    return SWEEP_OK;
}

sweep_status sweep_set_mesh(sweep_ctx* c, int64_t n_cells, const double* volume, int64_t n_faces,
                            const int32_t* face_cells, const double* area, const double* normal, const uint8_t* flags,
                            int32_t n_meshes, const int64_t* mesh_cell_offset) {
    if (!c) return SWEEP_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (n_cells < 1 || n_cells >= (1ll << 30)) return bad(c, "n_cells must be in [1, 2^30)");
    if (n_faces < 0) return bad(c, "n_faces < 0");
    if (!volume || (n_faces > 0 && (!face_cells || !area || !normal || !flags))) return bad(c, "null mesh array");
    std::vector<int64_t> off;
    if (n_meshes <= 0 || !mesh_cell_offset) off = {0, n_cells};
    else {
        off.assign(mesh_cell_offset, mesh_cell_offset + n_meshes + 1);
        if (off[0] != 0 || off.back() != n_cells) return bad(c, "mesh_cell_offset must run from 0 to n_cells");
        for (int i = 0; i < n_meshes; ++i)
            if (off[i + 1] <= off[i]) return bad(c, "mesh_cell_offset must be increasing");
    }
    int64_t S = 0, NB = 0;
    for (int64_t f = 0; f < n_faces; ++f) {
        S += face_cells[2 * f + 1] >= 0 ? 2 : 1;
        NB += (flags[f] & SWEEP_FACE_BOUNDARY) ? 1 : 0;
    }
    if (S >= (1ll << 32) - 64) return bad(c, "too many face sides (>= 2^32)");
    // drop everything tied to the previous mesh
    cudaStreamSynchronize(c->st);
    free_levels(c->lev);
    free_levels(c->adj_lev);
    free_solution(c);
    free_material(c);
    free_mesh(c->mesh);
    c->has_mesh = false;
    // upload and validate
    double *d_vol = nullptr, *d_area = nullptr, *d_normal = nullptr;
    int32_t *d_fc = nullptr, *d_tmp = nullptr;
    uint8_t* d_flags = nullptr;
    int64_t* d_off = nullptr;
    int* d_bad = nullptr;
    int64_t F1 = n_faces > 0 ? n_faces : 1;
    auto cleanup = [&]() {
        cudaFree(d_area); cudaFree(d_normal); cudaFree(d_fc); cudaFree(d_tmp); cudaFree(d_flags);
        cudaFree(d_off); cudaFree(d_bad);
    };
#define CKM(x, what) do { cudaError_t _e = (x); if (_e != cudaSuccess) { cleanup(); cudaFree(d_vol); return cuda_status(c, _e, what); } } while (0)
    CKM(cudaMalloc(&d_vol, sizeof(double) * n_cells), "alloc volume");
    CKM(cudaMalloc(&d_area, sizeof(double) * F1), "alloc area");
    CKM(cudaMalloc(&d_normal, sizeof(double) * 3 * F1), "alloc normal");
    CKM(cudaMalloc(&d_fc, sizeof(int32_t) * 2 * F1), "alloc faces");
    CKM(cudaMalloc(&d_flags, F1), "alloc flags");
    CKM(cudaMalloc(&d_off, sizeof(int64_t) * off.size()), "alloc offsets");
    CKM(cudaMalloc(&d_bad, sizeof(int)), "alloc");
    CKM(cudaMalloc(&d_tmp, sizeof(int32_t) * ((n_cells > n_faces ? n_cells : n_faces) + 2)), "alloc");
    CKM(cudaMemcpyAsync(d_vol, volume, sizeof(double) * n_cells, cudaMemcpyHostToDevice, c->st), "upload");
    if (n_faces > 0) {
        CKM(cudaMemcpyAsync(d_area, area, sizeof(double) * n_faces, cudaMemcpyHostToDevice, c->st), "upload");
        CKM(cudaMemcpyAsync(d_normal, normal, sizeof(double) * 3 * n_faces, cudaMemcpyHostToDevice, c->st), "upload");
        CKM(cudaMemcpyAsync(d_fc, face_cells, sizeof(int32_t) * 2 * n_faces, cudaMemcpyHostToDevice, c->st), "upload");
        CKM(cudaMemcpyAsync(d_flags, flags, n_faces, cudaMemcpyHostToDevice, c->st), "upload");
    }
    CKM(cudaMemcpyAsync(d_off, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, c->st), "upload");
    CKM(cudaMemsetAsync(d_bad, 0, sizeof(int), c->st), "init");
    CKM(launch_validate_mesh(n_cells, n_faces, d_vol, d_fc, d_area, d_normal, d_flags, d_off, (int)off.size() - 1,
                             d_bad, c->st), "validate mesh");
    int hbad = 0;
    CKM(cudaMemcpyAsync(&hbad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->st), "validate mesh");
    CKM(cudaStreamSynchronize(c->st), "validate mesh");
    if (hbad) {
        cleanup();
        cudaFree(d_vol);
        char buf[160];
        snprintf(buf, sizeof buf,
                 "invalid mesh (flags %d: 1 cell index, 2 face flags, 4 area, 8 normal, 16 volume, 32 face crosses "
                 "meshes, 64 self face)", hbad);
        return bad(c, buf);
    }
    DevMesh& m = c->mesh;
    m.N = n_cells;
    m.F = n_faces;
    m.S = S;
    m.NB = NB;
    m.vol = d_vol;
    m.mesh_off = off;
    CKM(cudaMalloc(&m.rowptr, sizeof(uint32_t) * (n_cells + 1)), "alloc rows");
    CKM(cudaMalloc(&m.side, sizeof(int4) * (S > 0 ? S : 1) + 64 * sizeof(int4)), "alloc sides");
    CKM(cudaMalloc(&m.side64, sizeof(d4) * (S > 0 ? S : 1)), "alloc sides");
    CKM(cudaMalloc(&m.side_lo, sizeof(float4) * (S > 0 ? S : 1)), "alloc sides");
    CKM(cudaMalloc(&m.nbr_rows, sizeof(int2) * (S > 0 ? S : 1)), "alloc sides");
    CKM(cudaMalloc(&m.twin, sizeof(uint32_t) * (S > 0 ? S : 1)), "alloc sides");
    CKM(launch_build_csr(m, d_fc, d_area, d_normal, d_flags, d_tmp, c->st), "build CSR");
    CKM(cudaStreamSynchronize(c->st), "build CSR");
#undef CKM
    cleanup();
    c->has_mesh = true;
    return SWEEP_OK;
}

sweep_status sweep_set_directions(sweep_ctx* c, int32_t n_dir, const double* omega, const double* weight) {
    if (!c) return SWEEP_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (n_dir < 1 || n_dir > 1024) return bad(c, "n_dir must be in [1, 1024]");
    if (!omega || !weight) return bad(c, "null direction array");
    double ws = 0.0;
    for (int d = 0; d < n_dir; ++d) {
        double x = omega[3 * d], y = omega[3 * d + 1], z = omega[3 * d + 2];
        double n2 = x * x + y * y + z * z;
        if (!(std::fabs(n2 - 1.0) <= 2.5e-9)) return bad(c, "direction is not a unit vector");
        if (!(weight[d] > 0.0) || !std::isfinite(weight[d])) return bad(c, "direction weight must be > 0");
        ws += weight[d];
    }
    if (!(std::fabs(ws - FOURPI) <= 1e-12 * FOURPI)) return bad(c, "direction weights must sum to 4pi");
    cudaStreamSynchronize(c->st);
    dfree(c->om64); dfree(c->w64); dfree(c->om32); dfree(c->om32lo);
    free_levels(c->lev);
    free_levels(c->adj_lev);
    free_solution(c);
    std::vector<float4> o32(n_dir), o32lo(n_dir);
    for (int d = 0; d < n_dir; ++d) {
        const double* w = omega + 3 * d;
        o32[d] = make_float4((float)w[0], (float)w[1], (float)w[2], (float)weight[d]);
        o32lo[d] = make_float4((float)(w[0] - (double)o32[d].x), (float)(w[1] - (double)o32[d].y),
                               (float)(w[2] - (double)o32[d].z), 0.f);
    }
    CK(cudaMalloc(&c->om64, sizeof(double) * 3 * n_dir), "alloc directions");
    CK(cudaMalloc(&c->w64, sizeof(double) * n_dir), "alloc directions");
    CK(cudaMalloc(&c->om32, sizeof(float4) * n_dir), "alloc directions");
    CK(cudaMalloc(&c->om32lo, sizeof(float4) * n_dir), "alloc directions");
    CK(cudaMemcpyAsync(c->om64, omega, sizeof(double) * 3 * n_dir, cudaMemcpyHostToDevice, c->st), "upload");
    CK(cudaMemcpyAsync(c->w64, weight, sizeof(double) * n_dir, cudaMemcpyHostToDevice, c->st), "upload");
    CK(cudaMemcpyAsync(c->om32, o32.data(), sizeof(float4) * n_dir, cudaMemcpyHostToDevice, c->st), "upload");
    CK(cudaMemcpyAsync(c->om32lo, o32lo.data(), sizeof(float4) * n_dir, cudaMemcpyHostToDevice, c->st), "upload");
    CK(cudaStreamSynchronize(c->st), "upload directions");
    c->D = n_dir;
    c->wsum = ws;
    c->has_dirs = true;
    return SWEEP_OK;
}

static sweep_status set_material_impl(sweep_ctx* c, int32_t G, const double* ka, const double* ks, const double* em,
                                      const double* bc, bool dev) {
    if (!c) return SWEEP_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (!c->has_mesh) return bad(c, "set the mesh first");
    if (G < 1 || G > 8) return bad(c, "n_groups must be in [1, 8]");
    if (!ka || !em) return bad(c, "kappa_abs and emissivity are required");
    const int64_t NG = c->mesh.N * (int64_t)G;
    const int64_t NBG = c->mesh.NB * (int64_t)G;
    bool scat = false;
    if (!dev) {
        for (int64_t i = 0; i < NG; ++i) {
            if (!(ka[i] >= 0.0) || !std::isfinite(ka[i])) return bad(c, "kappa_abs must be finite and >= 0");
            if (!(em[i] >= 0.0) || !std::isfinite(em[i])) return bad(c, "emissivity must be finite and >= 0");
            if (ks) {
                if (!(ks[i] >= 0.0) || !std::isfinite(ks[i])) return bad(c, "kappa_scat must be finite and >= 0");
                if (ks[i] > 0.0) scat = true;
            }
        }
        if (bc)
            for (int64_t i = 0; i < NBG; ++i)
                if (!(bc[i] >= 0.0) || !std::isfinite(bc[i])) return bad(c, "boundary_inflow must be finite and >= 0");
    }
    cudaStreamSynchronize(c->st);
    free_material(c);
    cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    size_t nb = sizeof(double) * (NG > 0 ? NG : 1);
    CK(cudaMalloc(&c->ka, nb), "alloc material");
    CK(cudaMalloc(&c->em, nb), "alloc material");
    CK(cudaMemcpyAsync(c->ka, ka, sizeof(double) * NG, kind, c->st), "upload material");
    CK(cudaMemcpyAsync(c->em, em, sizeof(double) * NG, kind, c->st), "upload material");
    if (ks) {
        CK(cudaMalloc(&c->ks, nb), "alloc material");
        CK(cudaMemcpyAsync(c->ks, ks, sizeof(double) * NG, kind, c->st), "upload material");
        if (dev) scat = true;  // not inspected on the host; a zero array costs one extra sweep
    }
    if (bc && NBG > 0) {
        CK(cudaMalloc(&c->bc, sizeof(double) * NBG), "alloc boundary inflow");
        CK(cudaMemcpyAsync(c->bc, bc, sizeof(double) * NBG, kind, c->st), "upload boundary inflow");
    }
    if (!dev) CK(cudaStreamSynchronize(c->st), "upload material");
    c->G = G;
    c->has_scat = scat;
    c->has_mat = true;
    return SWEEP_OK;
}

sweep_status sweep_set_material(sweep_ctx* c, int32_t G, const double* ka, const double* ks, const double* em,
                                const double* bc) {
    return set_material_impl(c, G, ka, ks, em, bc, false);
}

sweep_status sweep_set_material_dev(sweep_ctx* c, int32_t G, const double* ka, const double* ks, const double* em,
                                    const double* bc) {
    return set_material_impl(c, G, ka, ks, em, bc, true);
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
namespace {

// scheme (b) tables of the cached levels (empty in scheme (a))
DcTabs dc_tabs(sweep_ctx* c, const Levels& L) {
    DcTabs t;
    if (L.transport > 0) {
        t.mask = L.dc_mask;
        t.share64 = L.dc_share64;
        t.twin = c->mesh.twin;
    }
    return t;
}

// Form of the assembled operator a solve with these options sweeps over (OPF_NONE: it reads the mesh).
int wanted_format(sweep_ctx* c, const Levels& L, const sweep_opts* o, int prec) {
    if (prec != 32 || !o || o->geometry_only || o->schedule == SWEEP_SCHED_PLAIN) return OPF_NONE;
    const int G = c->G;
    const bool pk_ok = (G == 1 || G == 2 || G == 4) && (uint64_t)c->mesh.N * (uint64_t)L.nd <= (1ull << 31);
    // scheme (b) (its shares live in the packets) and the EXP law have the packed form only; otherwise
    // the mesh-row kernel
    if (L.transport > 0 || o->law != SWEEP_LAW_BALANCE) return pk_ok ? OPF_PACKETS : OPF_NONE;
    if (pk_ok && (o->op_format == SWEEP_OP_PACKETS || (o->op_format == SWEEP_OP_AUTO && o->lanes_per_task == 0)))
        return OPF_PACKETS;
    return OPF_LINES;
}

// device memory for an operator of `bytes`, keeping a margin for the solve buffers allocated later
bool op_fits(size_t bytes) {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    return bytes + (size_t)(2ull << 30) <= free_b;
}

// Plans and writes a packed operator of the levels L (transposed: the adjoint's), growing its buffers
// when device memory allows; false when it does not fit or a task has more entries than a packet holds.
bool build_packed(sweep_ctx* c, Levels& L, PackedOp& P, bool transposed) {
    int64_t n_pk = 0;
    if (pack_plan(c->mesh, L, P, transposed, c->om64, c->om32, c->om32lo, c->st, &n_pk) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    c->launches += 2;  // count pass, scan
    bool ok = n_pk >= 0;  // < 0: a task has more entries than a packet holds
    if (ok && n_pk > P.cap) {
        dfree(P.pk);
        dfree(P.meta);
        P.cap = 0;
        const int64_t cap = n_pk + n_pk / 16 + 64;
        ok = op_fits((size_t)cap * 520) && cudaMalloc(&P.pk, (size_t)cap * 512) == cudaSuccess &&
             cudaMalloc(&P.meta, (size_t)cap * 8) == cudaSuccess;
        if (ok) P.cap = cap;
        else {
            cudaGetLastError();
            dfree(P.pk);
            dfree(P.meta);
        }
    }
    if (!ok) return false;
    if (pack_write(c->mesh, L, P, transposed, c->om64, c->om32, c->om32lo, c->st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    c->launches += 1;  // write pass
    P.n_pk = n_pk;
    return true;
}

// The packed transposed operator of the cached levels for the FP32 adjoint sweep (2G = 2 or 4 split
// groups, the packed kernel's widths), built once per levelisation; without it (memory, rows longer
// than a packet, other group counts) the transposed sweep reads the mesh rows.
sweep_status ensure_transposed(sweep_ctx* c, Levels& L, const sweep_opts* o, int prec, float* t_ms) {
    const int G2 = 2 * c->G;
    if (prec != 32 || (o && (o->geometry_only || o->schedule == SWEEP_SCHED_PLAIN)) || (G2 != 2 && G2 != 4) ||
        (uint64_t)c->mesh.N * (uint64_t)L.nd > (1ull << 31) || L.transport > 0)
        return SWEEP_OK;
    if (L.pkt.valid) return SWEEP_OK;
    ScopedEvent e0, e1;
    cudaEventRecord(e0, c->st);
    L.pkt.valid = build_packed(c, L, L.pkt, true);
    cudaEventRecord(e1, c->st);
    CK(cudaEventSynchronize(e1), "assemble transposed operator");
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (t_ms) *t_ms += ms;
    return SWEEP_OK;
}

// Assembles the transport operator of the levelised directions in the form the solve sweeps over
// (128-byte lines or packets), when device memory allows; otherwise the FP32 sweep reads the mesh
// geometry directly. Built once per levelisation and kept while the form stays the same.
sweep_status ensure_operator(sweep_ctx* c, Levels& L, const sweep_opts* o, int prec, float* t_ms) {
    int want = wanted_format(c, L, o, prec);
    if (want == OPF_NONE || (L.op_valid && L.op_format == want)) return SWEEP_OK;
    L.op_valid = false;
    ScopedEvent e0, e1;
    cudaEventRecord(e0, c->st);
    if (want == OPF_PACKETS) {
        dfree(L.op);  // the other form's buffer
        L.op_bytes = 0;
        if (build_packed(c, L, L.pk, false)) {
            c->launches += 1;  // the level table
            L.op_format = OPF_PACKETS;
            L.op_valid = true;
        } else {
            want = OPF_LINES;
        }
    }
    if (want == OPF_LINES) {
        dfree(L.pk.pk);
        dfree(L.pk.meta);
        L.pk.cap = 0;
        const int64_t tasks = L.h_lev_chunk.empty() ? 0 : L.h_lev_chunk.back() * 32;
        const size_t bytes = (size_t)tasks * 128;
        bool ok = true;
        if (bytes > L.op_bytes) {
            dfree(L.op);
            L.op_bytes = 0;
            ok = op_fits(bytes) && cudaMalloc(&L.op, bytes) == cudaSuccess;
            if (ok) L.op_bytes = bytes;
            else {
                cudaGetLastError();
                L.op = nullptr;
            }
        }
        if (ok) {
            CKL(build_operator(c->mesh, L, c->om64, c->om32, c->om32lo, c->st), "assemble operator");
            L.op_format = OPF_LINES;
            L.op_valid = true;
        }
    }
    cudaEventRecord(e1, c->st);
    CK(cudaEventSynchronize(e1), "assemble operator");
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (t_ms) *t_ms = ms;
    return SWEEP_OK;
}

// Levels of every direction in the dependency graph of the requested transport scheme (without options:
// whatever scheme is cached, else scheme (a)).
sweep_status ensure_levels(sweep_ctx* c, const sweep_opts* o, float* t1, float* t2) {
    const int tr = o ? o->transport : (c->lev.valid ? c->lev.transport : 0);
    if (c->lev.valid && !(o && o->relevel) && c->lev.nd == c->D && c->lev.d0 == 0 && c->lev.transport == tr)
        return SWEEP_OK;
    c->lev.op_valid = false;
    c->lev.pkt.valid = false;
    return run_levelise(c, c->lev, 0, c->D, budget_of(o), t1, t2, tr);
}

sweep_status ensure_solution(sweep_ctx* c, int prec, bool two) {
    SolveBuf& b = c->sb;
    const size_t es = prec == 64 ? 8 : 4;
    const size_t bytes = es * (size_t)c->mesh.N * c->D * c->G;
    if (b.bytes != bytes || b.prec != prec || b.N != c->mesh.N || b.nd != c->D || b.G != c->G) {
        dfree(b.I[0]);
        dfree(b.I[1]);
        b = SolveBuf();
        CK(cudaMalloc(&b.I[0], bytes > 0 ? bytes : 4), "alloc intensities");
        CK(cudaMemsetAsync(b.I[0], 0, bytes, c->st), "init intensities");
        b.bytes = bytes;
        b.prec = prec;
        b.N = c->mesh.N;
        b.nd = c->D;
        b.G = c->G;
    }
    if (two && !b.I[1]) {
        CK(cudaMalloc(&b.I[1], bytes > 0 ? bytes : 4), "alloc intensities");
        CK(cudaMemsetAsync(b.I[1], 0, bytes, c->st), "init intensities");
        b.sign[1] = 0;
    }
    return SWEEP_OK;
}

sweep_status ensure_mean(sweep_ctx* c, int prec) {
    const size_t bytes = (prec == 64 ? 8 : 4) * (size_t)c->mesh.N * c->D * c->G;
    if (c->Imean && c->imean_bytes == bytes) return SWEEP_OK;
    dfree(c->Imean);
    c->imean_bytes = 0;
    CK(cudaMalloc(&c->Imean, bytes > 0 ? bytes : 4), "alloc cell means");
    c->imean_bytes = bytes;
    return SWEEP_OK;
}

double read_max(sweep_ctx* c) {
    unsigned long long v = 0;
    cudaMemcpyAsync(&v, c->dmax, sizeof v, cudaMemcpyDeviceToHost, c->st);
    cudaStreamSynchronize(c->st);
    double d;
    memcpy(&d, &v, sizeof d);
    return d;
}

// choose schedule and block size: time one sweep per candidate (results are identical for all)
struct LaunchCfg {
    int sched, threads, lanes, bpsm;
};

// choose the batched-sweep configuration: time one sweep per candidate (results are identical for all)
sweep_status autotune(sweep_ctx* c, int prec, const void* cm, const float* bc32, const sweep_opts* o, LaunchCfg* out) {
    const int fmt = (prec == 32 && c->lev.op_valid && !(o && o->geometry_only)) ? c->lev.op_format : OPF_NONE;
    int* t4 = c->tuned[prec == 64][c->G][fmt];
    if (t4[0]) {
        *out = LaunchCfg{t4[0], t4[1], t4[2], t4[3]};
        return SWEEP_OK;
    }
    std::vector<LaunchCfg> cand;
    if (fmt == OPF_PACKETS) {
        // packets per warp step: one (lanes 32) or two (lanes 64); the level-synchronous form with two
        // (three resident blocks per SM: fewer polling warps compete with the ones that have work)
        cand.push_back({SWEEP_SCHED_DATAFLOW, 256, 64, 0});
        cand.push_back({SWEEP_SCHED_DATAFLOW, 256, 64, 3});
        cand.push_back({SWEEP_SCHED_DATAFLOW, 256, 32, 0});
        cand.push_back({SWEEP_SCHED_LEVEL, 256, 64, 0});
    } else if (fmt == OPF_LINES) {
        // 8 lanes per task (4 tasks per warp step) and 4 lanes per task (8 tasks per step)
        cand.push_back({SWEEP_SCHED_DATAFLOW, 256, 8, 0});
        cand.push_back({SWEEP_SCHED_DATAFLOW, 256, 16, 0});
        cand.push_back({SWEEP_SCHED_DATAFLOW, 256, 4, 0});
        cand.push_back({SWEEP_SCHED_LEVEL, 256, 8, 0});
    } else {
        for (int s : {SWEEP_SCHED_LEVEL, SWEEP_SCHED_DATAFLOW})
            for (int t : {128, 256})
                for (int l : {1, 2, 4, 8, 16}) cand.push_back({s, t, l, 0});
    }
    float best = 1e30f;
    LaunchCfg bc = cand[0];
    SolveBuf& b = c->sb;
    const int tb = (b.last == 0 && b.I[1]) ? 1 : 0;
    auto time_one = [&](const LaunchCfg& k, float* ms) {
        const int parity = !b.sign[tb];
        SweepArgs a = make_args(c, c->lev, prec, cm, b.I[tb], nullptr, c->G, parity, 0, 0, o);
        a.debug_stall = 0;
        sweep_status st = run_sweep(c, c->lev, prec, k.sched, k.threads, k.lanes, k.bpsm, a, bc32, ms);
        if (st == SWEEP_OK) b.sign[tb] = parity;
        return st;
    };
    // one untimed sweep first (caches, first touch of the buffers), then the best of two per candidate
    float warm = 0;
    sweep_status st0 = time_one(cand[0], &warm);
    if (st0 != SWEEP_OK) return st0;
    for (const LaunchCfg& k : cand) {
        float m = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            float ms = 0;
            sweep_status st = time_one(k, &ms);
            if (st != SWEEP_OK) return st;
            m = std::min(m, ms);
        }
        if (m < best) {
            best = m;
            bc = k;
        }
    }
    t4[0] = bc.sched;
    t4[1] = bc.threads;
    t4[2] = bc.lanes;
    t4[3] = bc.bpsm;
    *out = bc;
    return SWEEP_OK;
}

// device scratch freed at scope exit
template <typename T>
struct DevBuf {
    T* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};
__global__ void k_bc_to_f32(const double* in, int64_t n, float* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

// the FP32 copy of the boundary inflow, kept in the context from the first FP32 solve after set_material
sweep_status ensure_bc32(sweep_ctx* c) {
    if (c->bc32_ready) return SWEEP_OK;
    const int64_t n = c->mesh.NB * c->G;
    if (!c->bc32) CK(cudaMalloc(&c->bc32, sizeof(float) * (n > 0 ? n : 1)), "alloc boundary inflow");
    k_bc_to_f32<<<nblocks256(n), 256, 0, c->st>>>(c->bc, n, c->bc32);
    ++c->launches;
    CK(cudaGetLastError(), "boundary inflow");
    c->bc32_ready = true;
    return SWEEP_OK;
}

sweep_status solve_impl(sweep_ctx* c, const sweep_opts* opts_in, double* J_out, double* Gam_out, bool dev,
                        sweep_stats* stats) {
    if (!c) return SWEEP_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (!c->has_mesh || !c->has_dirs || !c->has_mat) return bad(c, "set mesh, directions and material first");
    sweep_opts o;
    if (opts_in) o = *opts_in;
    else sweep_default_opts(&o);
    if (o.law != SWEEP_LAW_BALANCE && o.law != SWEEP_LAW_EXP) return bad(c, "unsupported law");
    const bool plain = o.schedule == SWEEP_SCHED_PLAIN;
    const int prec = plain ? 64 : (o.precision == 64 ? 64 : 32);
    if (o.precision != 32 && o.precision != 64) return bad(c, "precision must be 32 or 64");
    if (o.block_threads != 0 && o.block_threads != 128 && o.block_threads != 256)
        return bad(c, "block_threads must be 0, 128 or 256");
    if (o.lanes_per_task < 0 || o.lanes_per_task > 16 || (o.lanes_per_task & (o.lanes_per_task - 1)))
        return bad(c, "lanes_per_task must be 0, 1, 2, 4, 8 or 16");
    sweep_stats S;
    memset(&S, 0, sizeof S);
    const int64_t launches0 = c->launches;
    ScopedEvent t0, t1;
    cudaEventRecord(t0, c->st);
    if (o.op_format < SWEEP_OP_AUTO || o.op_format > SWEEP_OP_PACKETS) return bad(c, "op_format must be 0, 1 or 2");
    if (o.packets_per_step < 0 || o.packets_per_step > 2) return bad(c, "packets_per_step must be 0, 1 or 2");
    if (o.transport < 0 || o.transport > 8) return bad(c, "transport must be 0 (scheme (a)) or 1..8 (scheme (b))");
    float tc = 0, tl = 0, top = 0;
    sweep_status s = ensure_levels(c, &o, &tc, &tl);
    if (s != SWEEP_OK) return s;
    s = ensure_operator(c, c->lev, &o, prec, &top);
    if (s != SWEEP_OK) return s;
    S.t_ms[0] = tc;
    S.t_ms[1] = tl;
    S.t_ms[5] = top;
    const int64_t N = c->mesh.N;
    const int G = c->G, D = c->D;
    const size_t NG = (size_t)N * G;
    const bool has_pbc = c->mesh.n_pcells > 0;
    s = ensure_ng(c, NG);
    if (s != SWEEP_OK) return s;
    s = ensure_cm(c, NG);
    if (s != SWEEP_OK) return s;
    s = ensure_solution(c, prec, has_pbc);
    if (s != SWEEP_OK) return s;
    if (o.law) {
        s = ensure_mean(c, prec);
        if (s != SWEEP_OK) return s;
    }
    // partial sums: one pair per 256-thread block of the tallies, one pair per periodic or boundary cell
    const int nblk = nblocks256(NG);
    int64_t npart = nblk + 1;
    if (c->mesh.n_pcells > npart) npart = c->mesh.n_pcells;
    if (c->mesh.n_bcells > npart) npart = c->mesh.n_bcells;
    s = ensure_partial(c, (int)npart);
    if (s != SWEEP_OK) return s;
    const float* bc32 = nullptr;
    if (prec == 32 && c->bc) {
        s = ensure_bc32(c);
        if (s != SWEEP_OK) return s;
        bc32 = c->bc32;
    }
    SolveBuf& b = c->sb;
    const void* cm = prec == 64 ? (const void*)c->cm64 : (const void*)c->cm32;
    int sched = o.schedule, threads = o.block_threads ? o.block_threads : 256;
    int lanes = o.lanes_per_task ? o.lanes_per_task : 4;
    int bpsm = o.blocks_per_sm;
    // the EXP law: no tuning, the dataflow schedule (packets: two per warp step)
    if (!plain && sched == SWEEP_SCHED_AUTO && o.law) sched = SWEEP_SCHED_DATAFLOW;
    if (!plain && sched == SWEEP_SCHED_AUTO) {
        CKL(launch_prep_material(N, G, c->mesh.vol, c->ka, c->ks, c->em, nullptr, prec == 32 ? c->cm32 : nullptr,
                                prec == 64 ? c->cm64 : nullptr, c->st), "prep");
        LaunchCfg best;
        s = autotune(c, prec, cm, bc32, &o, &best);
        sched = best.sched;
        const int tt = best.threads, tl = best.lanes;
        if (!o.blocks_per_sm) bpsm = best.bpsm;
        if (s != SWEEP_OK) return s;
        if (!o.block_threads) threads = tt;
        if (!o.lanes_per_task) lanes = tl;
    }
    // the packed operator's kernel has whole warps per packet: lanes = 32 x packets per warp step
    const bool packed = prec == 32 && !o.geometry_only && c->lev.op_valid && c->lev.op_format == OPF_PACKETS;
    if (!plain && packed) {
        if (o.packets_per_step) lanes = 32 * o.packets_per_step;
        else if (lanes < 32) lanes = 64;
    }
    // the periodic inflow of the first sweep: the previous solve's intensities or zeros
    int prev = -1;
    if (has_pbc) {
        c->ptab.ready = false;
        const DcTabs dct = dc_tabs(c, c->lev);
        CK(build_periodic_table(c->mesh, D, c->om64, c->w64, &c->ptab, c->st, &dct), "periodic weights");
        c->launches += 3;
        if (o.warm_start && b.last >= 0) prev = b.last;
        else {
            prev = b.last >= 0 ? b.last : 1;
            CK(cudaMemsetAsync(b.I[prev], 0, b.bytes, c->st), "clear periodic inflow");
            b.sign[prev] = 0;
        }
        CK(cudaMemsetAsync(c->jn, 0, sizeof(double) * NG, c->st), "init");
        if (o.warm_start && b.last >= 0) {
            CK(cudaMemsetAsync(c->dmax, 0, sizeof(unsigned long long), c->st), "init");
            CKL(launch_periodic_source(prec, c->mesh, b.I[prev], G, D, c->om64, c->w64, c->jn1, c->jn, c->dmax,
                                      c->partial, nblk, c->st, &c->ptab), "periodic source");
            std::swap(c->jn, c->jn1);
        }
    }
    S.schedule_used = sched;
    S.lanes_used = lanes;
    S.threads_used = threads;
    S.blocks_per_sm_used = bpsm;
    int it_pbc = 0, it_scat_total = 0, n_sweeps = 0;
    bool conv_pbc = !has_pbc, conv_scat = !c->has_scat;
    double res_pbc = 0.0, res_pbc_mean = 0.0, res_scat = 0.0;
    float t_sweep = 0.f;
    int cur = has_pbc ? (prev == 0 ? 1 : 0) : 0;
    ScopedEvent u0, u1;
    float t_other = 0.f;
    bool graphed = false;
    // Sec. 2.7's fused loops: one source-iteration sweep per periodic iteration, J carried over
    const bool fused = o.fused_loops && has_pbc && c->has_scat;
    if (o.use_graph && !plain && !o.debug_stall && (has_pbc != c->has_scat || fused)) {
        // what stays fixed over the iterations: the source without scattering, J_old before Alg. 1
        if (has_pbc && !fused)
            CKL(launch_prep_material(N, G, c->mesh.vol, c->ka, c->ks, c->em, nullptr, prec == 32 ? c->cm32 : nullptr,
                                    prec == 64 ? c->cm64 : nullptr, c->st), "prep");
        else
            CK(cudaMemsetAsync(c->Jold, 0, sizeof(double) * NG, c->st), "init");
        LoopState ls;
        ls.cur = cur;
        ls.prev = prev;
        ls.conv_pbc = conv_pbc;
        ls.conv_scat = conv_scat;
        s = graph_loop(c, o, prec, cm, bc32, sched, threads, lanes, bpsm, nblk, ls, &graphed);
        if (s != SWEEP_OK) return s;
        if (graphed) {
            cur = ls.cur;
            prev = ls.prev;
            it_pbc = ls.it_pbc;
            it_scat_total = ls.it_scat_total;
            n_sweeps = ls.n_sweeps;
            conv_pbc = ls.conv_pbc;
            conv_scat = ls.conv_scat;
            res_pbc = ls.res_pbc;
            res_pbc_mean = ls.res_pbc_mean;
            res_scat = ls.res_scat;
            t_sweep = ls.t_sweep;
            t_other = ls.t_other;
        }
    }
    S.graph_used = graphed ? 1 : 0;
    for (; !graphed;) {
        if (!fused || it_pbc == 0) CK(cudaMemsetAsync(c->Jold, 0, sizeof(double) * NG, c->st), "init");
        int it_scat = 0;
        for (;;) {
            CKL(launch_prep_material(N, G, c->mesh.vol, c->ka, c->ks, c->em, c->has_scat ? c->Jold : nullptr,
                                    prec == 32 ? c->cm32 : nullptr, prec == 64 ? c->cm64 : nullptr, c->st), "prep");
            const int parity = !b.sign[cur];
            SweepArgs a = make_args(c, c->lev, prec, cm, b.I[cur], has_pbc ? b.I[prev] : nullptr, G, parity, 0, 0, &o);
            a.debug_stall = o.debug_stall && n_sweeps == 0;
            s = run_sweep(c, c->lev, prec, plain ? SWEEP_SCHED_PLAIN : sched, threads, lanes, bpsm, a, bc32,
                          &t_sweep);
            if (s != SWEEP_OK) return s;
            b.sign[cur] = parity;
            ++n_sweeps;
            ++it_scat;
            // without scattering nothing inside the iteration needs J: the final tally below computes it
            if (!c->has_scat) break;
            cudaEventRecord(u0, c->st);
            CKL(launch_tally(prec, o.law ? c->Imean : b.I[cur], N, G, D, 0, c->w64, c->wsum, c->mesh.vol, c->ka,
                            c->em, c->J, c->Gam, c->partial, nblk, c->st), "tally");
            CK(cudaMemsetAsync(c->dmax, 0, sizeof(unsigned long long), c->st), "init");
            CKL(launch_scat_residual(NG, c->J, c->Jold, c->dmax, c->st), "scattering residual");
            cudaEventRecord(u1, c->st);
            res_scat = read_max(c);
            float tt = 0;
            cudaEventElapsedTime(&tt, u0, u1);
            t_other += tt;
            if (fused) {
                conv_scat = res_scat <= o.tol_scat;
                break;
            }
            if (res_scat <= o.tol_scat) { conv_scat = true; break; }
            if (it_scat >= o.max_it_scat) { conv_scat = false; break; }
        }
        it_scat_total += it_scat;
        ++it_pbc;
        if (!has_pbc) break;
        cudaEventRecord(u0, c->st);
        CK(cudaMemsetAsync(c->dmax, 0, sizeof(unsigned long long), c->st), "init");
        CKL(launch_periodic_source(prec, c->mesh, b.I[cur], G, D, c->om64, c->w64, c->jn1, c->jn, c->dmax, c->partial,
                                  nblk, c->st, &c->ptab), "periodic source");
        CKL(launch_reduce_sum(c->partial, (int)c->mesh.n_pcells, c->red + 2, c->st), "reduce");
        cudaEventRecord(u1, c->st);
        res_pbc = read_max(c);
        double hred[2] = {0, 0};
        CK(cudaMemcpyAsync(hred, c->red + 2, sizeof hred, cudaMemcpyDeviceToHost, c->st), "read");
        CK(cudaStreamSynchronize(c->st), "read");
        float tt = 0;
        cudaEventElapsedTime(&tt, u0, u1);
        t_other += tt;
        res_pbc_mean = NG > 0 ? hred[0] / (double)NG : 0.0;
        std::swap(c->jn, c->jn1);
        prev = cur;
        cur = 1 - cur;
        if (fused) {
            conv_pbc = res_pbc < o.tol_pbc;
            if ((conv_pbc && conv_scat) || it_pbc >= o.max_it_pbc) break;
            continue;
        }
        if (res_pbc < o.tol_pbc) { conv_pbc = true; break; }
        if (it_pbc >= o.max_it_pbc) { conv_pbc = false; break; }
    }
    const int fin = has_pbc ? prev : cur;
    b.last = fin;
    // final tallies: absorbed/emitted from the last tally, escaped/injected over boundary cells
    CKL(launch_tally(prec, o.law ? c->Imean : b.I[fin], N, G, D, 0, c->w64, c->wsum, c->mesh.vol, c->ka, c->em, c->J,
                    c->Gam, c->partial, nblk, c->st), "tally");
    CKL(launch_reduce_sum(c->partial, nblocks256(NG), c->red, c->st), "reduce");
    if (c->mesh.n_bcells > 0) {
        const DcTabs dct = dc_tabs(c, c->lev);
        CKL(launch_boundary_tally(prec, c->mesh, b.I[fin], G, D, 0, c->om64, c->w64, c->bc, c->partial, nblk, c->st,
                                  &dct),
           "boundary tally");
        CKL(launch_reduce_sum(c->partial, (int)c->mesh.n_bcells, c->red + 2, c->st), "reduce");
    } else {
        CK(cudaMemsetAsync(c->red + 2, 0, 2 * sizeof(double), c->st), "init");
    }
    double hr[4];
    CK(cudaMemcpyAsync(hr, c->red, sizeof hr, cudaMemcpyDeviceToHost, c->st), "read tallies");
    cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (J_out) CK(cudaMemcpyAsync(J_out, c->J, sizeof(double) * NG, k, c->st), "copy J");
    if (Gam_out) CK(cudaMemcpyAsync(Gam_out, c->Gam, sizeof(double) * NG, k, c->st), "copy Gamma");
    cudaEventRecord(t1, c->st);
    CK(cudaStreamSynchronize(c->st), "solve");
    float ttot = 0;
    cudaEventElapsedTime(&ttot, t0, t1);
    S.absorbed = hr[0];
    S.emitted = hr[1];
    S.escaped = hr[2];
    S.injected = hr[3];
    double in = S.emitted + S.injected;
    S.defect = in > 0.0 ? (in - S.absorbed - S.escaped) / in : 0.0;
    S.it_scat = c->has_scat ? it_scat_total : 0;  // sweeps of the source iteration (none without scattering)
    S.it_pbc = it_pbc;
    S.n_sweeps = n_sweeps;
    S.kernel_used = c->last_kernel;
    S.res_scat = res_scat;
    S.res_pbc = res_pbc;
    S.res_pbc_mean = res_pbc_mean;
    S.t_ms[2] = t_sweep;
    S.t_ms[3] = t_other;
    S.t_ms[4] = ttot;
    S.updates = (double)N * D * G * n_sweeps;
    S.updates_per_s = ttot > 0 ? S.updates / (ttot * 1e-3) : 0.0;
    S.sweep_launches = plain ? 0 : n_sweeps;
    int dmaxv = 0;
    double dsum = 0;
    for (int d : c->lev.depth) {
        if (d > dmaxv) dmaxv = d;
        dsum += d;
    }
    S.depth_max = dmaxv;
    S.depth_mean = c->lev.depth.empty() ? 0.0 : dsum / c->lev.depth.size();
    S.kernel_launches = (int32_t)(c->launches - launches0);
    if (stats) *stats = S;
    return (conv_pbc && conv_scat) ? SWEEP_OK : SWEEP_NOT_CONVERGED;
}

sweep_status adjoint_impl(sweep_ctx* c, const sweep_opts* opts_in, const double* dlj, const double* dlg, double* gk_out,
                          double* ge_out, double* gks_out, bool dev, sweep_stats* stats) {
    if (!c) return SWEEP_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (!c->has_mesh || !c->has_dirs || !c->has_mat) return bad(c, "set mesh, directions and material first");
    if (c->G > 4) return bad(c, "the adjoint supports at most 4 groups");
    if (opts_in && opts_in->law != SWEEP_LAW_BALANCE) return bad(c, "the adjoint takes the BALANCE law");
    if (opts_in && opts_in->transport != 0) return bad(c, "the adjoint takes transport scheme (a)");
    if (!gk_out || !ge_out) return bad(c, "null gradient output");
    sweep_opts o;
    if (opts_in) o = *opts_in;
    else sweep_default_opts(&o);
    const bool plain = o.schedule == SWEEP_SCHED_PLAIN;
    const int prec = plain ? 64 : (o.precision == 64 ? 64 : 32);
    int sched = o.schedule == SWEEP_SCHED_AUTO ? SWEEP_SCHED_DATAFLOW : o.schedule;
    const int lanes = o.lanes_per_task ? o.lanes_per_task : 4;
    const int threads = o.block_threads ? o.block_threads : 256;
    const int64_t N = c->mesh.N;
    const int G = c->G, D = c->D;
    const size_t NG = (size_t)N * G;
    // With scattering or periodic faces the iterations couple all directions, and the kappa_s gradient
    // needs J: the forward state is then the solve itself (one batch of every direction), and the
    // transposed iteration lags both couplings by a pass.
    const bool scat = c->has_scat, pbc = c->mesh.n_pcells > 0;
    const bool coupled = scat || pbc || gks_out;
    if ((scat || pbc) && o.max_it_scat < 1) return bad(c, "max_it_scat must be >= 1");
    int B = (!coupled && o.dir_batch > 0 && o.dir_batch < D) ? o.dir_batch : D;
    sweep_stats S;
    memset(&S, 0, sizeof S);
    const int64_t launches0 = c->launches;
    ScopedEvent t0, t1;
    cudaEventRecord(t0, c->st);
    // device copies of the loss gradients and FP64 gradient accumulators
    DevBuf<double> b_dlj, b_dlg, b_gk, b_ge;
    cudaMemcpyKind kin = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (dlj) {
        CK(cudaMalloc(&b_dlj.p, sizeof(double) * (NG > 0 ? NG : 1)), "alloc");
        CK(cudaMemcpyAsync(b_dlj.p, dlj, sizeof(double) * NG, kin, c->st), "upload");
    }
    if (dlg) {
        CK(cudaMalloc(&b_dlg.p, sizeof(double) * (NG > 0 ? NG : 1)), "alloc");
        CK(cudaMemcpyAsync(b_dlg.p, dlg, sizeof(double) * NG, kin, c->st), "upload");
    }
    CK(cudaMalloc(&b_gk.p, sizeof(double) * (NG > 0 ? NG : 1)), "alloc");
    CK(cudaMalloc(&b_ge.p, sizeof(double) * (NG > 0 ? NG : 1)), "alloc");
    double *d_dlj = b_dlj.p, *d_dlg = b_dlg.p, *gk = b_gk.p, *ge = b_ge.p;
    CK(cudaMemsetAsync(gk, 0, sizeof(double) * NG, c->st), "init");
    CK(cudaMemsetAsync(ge, 0, sizeof(double) * NG, c->st), "init");
    DevBuf<double> b_gks, b_mu;
    if (gks_out) CK(cudaMalloc(&b_gks.p, sizeof(double) * (NG > 0 ? NG : 1)), "alloc");
    if (scat || pbc) {
        CK(cudaMalloc(&b_mu.p, sizeof(double) * (2 * NG > 0 ? 2 * NG : 1)), "alloc");
        CK(cudaMemsetAsync(b_mu.p, 0, sizeof(double) * 2 * NG, c->st), "init");
    }
    sweep_status s = SWEEP_OK;
    // forward state of the coupled problems: the solve (both iterations to their tolerances), whose
    // final sweep's intensities and J stay on the device
    int it_fwd = 0;
    bool conv_fwd = true;
    double res_fwd = 0.0;
    if (coupled) {
        sweep_stats fs;
        s = solve_impl(c, &o, nullptr, nullptr, true, &fs);
        if (s == SWEEP_NOT_CONVERGED) conv_fwd = false;
        else if (s != SWEEP_OK) return s;
        it_fwd = fs.n_sweeps;
        res_fwd = pbc ? fs.res_pbc : fs.res_scat;
    }
    s = ensure_cm(c, 2 * NG);
    if (s != SWEEP_OK) return s;
    // batch buffers
    const size_t es = prec == 64 ? 8 : 4;
    size_t bI = coupled ? es : es * (size_t)N * B * G, bL = es * (size_t)N * B * 2 * G;  // coupled: the solve's
    if (c->adj_bytes_I != bI || c->adj_bytes_L != bL) {
        dfree(c->adjI);
        dfree(c->adjL);
        CK(cudaMalloc(&c->adjI, bI > 0 ? bI : 4), "alloc adjoint batch");
        CK(cudaMalloc(&c->adjL, bL > 0 ? bL : 4), "alloc adjoint batch");
        c->adj_bytes_I = bI;
        c->adj_bytes_L = bL;
    }
    // fresh buffers each call: sign state starts at 0 after clearing; with periodic faces a second
    // lambda buffer holds the previous pass
    CK(cudaMemsetAsync(c->adjI, 0, bI, c->st), "init");
    CK(cudaMemsetAsync(c->adjL, 0, bL, c->st), "init");
    DevBuf<char> b_lam2;
    if (pbc) {
        CK(cudaMalloc(&b_lam2.p, bL > 0 ? bL : 4), "alloc adjoint batch");
        CK(cudaMemsetAsync(b_lam2.p, 0, bL, c->st), "init");
    }
    void* lbuf[2] = {c->adjL, b_lam2.p};
    int signI = 0, signL[2] = {0, 0}, kl = 0;
    const float* bc32 = nullptr;
    if (prec == 32 && c->bc) {
        sweep_status sb = ensure_bc32(c);
        if (sb != SWEEP_OK) return sb;
        bc32 = c->bc32;
    }
    float t_sweep = 0.f, tcl = 0.f, tlv = 0.f, tasm = 0.f, t_tr = 0.f;
    // the packed kernels take whole warps per packet: 32 lanes x packets per warp step; unless given, the
    // forward solve's autotuned choice for this mesh (one packet per step on narrow levels, two on wide)
    const int* tuned = c->tuned[0][G][OPF_PACKETS];
    const int pk_lanes = o.packets_per_step ? 32 * o.packets_per_step : (tuned[0] && tuned[2] >= 32 ? tuned[2] : 64);
    const int pk_bpsm = o.blocks_per_sm ? o.blocks_per_sm : (tuned[0] ? tuned[3] : 0);
    int n_sweeps = it_fwd, it_adj = 0;
    bool conv_adj = true;
    double res_adj = 0.0;
    for (int d0 = 0; d0 < D; d0 += B) {
        const int nb = (D - d0) < B ? (D - d0) : B;
        Levels* L;
        float a1 = 0, a2 = 0;
        if (nb == D) {
            s = ensure_levels(c, &o, &a1, &a2);
            if (s == SWEEP_OK) s = ensure_operator(c, c->lev, &o, prec, &tasm);
            if (s == SWEEP_OK) s = ensure_transposed(c, c->lev, &o, prec, &tasm);
            L = &c->lev;
        } else {
            s = run_levelise(c, c->adj_lev, d0, nb, budget_of(&o), &a1, &a2);
            L = &c->adj_lev;
        }
        if (s != SWEEP_OK) return s;
        tcl += a1;
        tlv += a2;
        const void* cm = prec == 64 ? (const void*)c->cm64 : (const void*)c->cm32;
        const void* Ifwd = c->adjI;
        if (coupled) {
            Ifwd = c->sb.I[c->sb.last];
        } else {
            // forward intensities of this batch (recomputed, not stored across batches)
            CKL(launch_prep_material(N, G, c->mesh.vol, c->ka, nullptr, c->em, nullptr,
                                    prec == 32 ? c->cm32 : nullptr, prec == 64 ? c->cm64 : nullptr, c->st), "prep");
            int pI = !signI;
            SweepArgs a = make_args(c, *L, prec, cm, c->adjI, nullptr, G, pI, 0, 0, &o);
            a.debug_stall = 0;
            s = run_sweep(c, *L, prec, plain ? SWEEP_SCHED_PLAIN : sched, threads, a.pk ? pk_lanes : lanes,
                          a.pk ? pk_bpsm : 0, a, bc32, &t_sweep);
            if (s != SWEEP_OK) return s;
            signI = pI;
            ++n_sweeps;
            ++it_fwd;
        }
        // transposed sweep with split non-negative sources (2G groups); with scattering or periodic faces
        // the transposed iteration: mu and the previous pass's lambda start at 0
        CKL(launch_prep_adjoint_src(N, G, c->mesh.vol, c->ka, scat ? c->ks : nullptr, d_dlj, d_dlg,
                                   prec == 32 ? c->cm32 : nullptr, prec == 64 ? c->cm64 : nullptr, c->st),
           "prep adjoint");
        for (;;) {
            int pL = !signL[kl];
            SweepArgs r = make_args(c, *L, prec, cm, lbuf[kl], pbc ? lbuf[1 - kl] : nullptr, 2 * G, pL, 1, 0, &o);
            r.debug_stall = 0;
            float t1 = 0.f;
            s = run_sweep(c, *L, prec, plain ? SWEEP_SCHED_PLAIN : sched, threads, r.pk ? pk_lanes : lanes,
                          r.pk ? pk_bpsm : 0, r, nullptr, &t1);
            t_sweep += t1;
            t_tr += t1;
            if (s != SWEEP_OK) return s;
            signL[kl] = pL;
            ++n_sweeps;
            ++it_adj;
            if (!scat && !pbc) break;
            CK(cudaMemsetAsync(c->dmax, 0, 2 * sizeof(unsigned long long), c->st), "init");
            CKL(launch_adjoint_mu(prec, lbuf[kl], N, G, D, c->mesh.vol, c->ka, scat ? c->ks : nullptr, d_dlj, d_dlg,
                                 b_mu.p, prec == 32 ? c->cm32 : nullptr, prec == 64 ? c->cm64 : nullptr, c->dmax,
                                 c->st),
               "transposed source");
            unsigned long long hm[2] = {0, 0};
            CK(cudaMemcpyAsync(hm, c->dmax, sizeof hm, cudaMemcpyDeviceToHost, c->st), "read");
            CK(cudaStreamSynchronize(c->st), "read");
            double dm, mm;
            memcpy(&dm, &hm[0], sizeof dm);
            memcpy(&mm, &hm[1], sizeof mm);
            res_adj = dm == 0.0 ? 0.0 : (mm > 0.0 ? dm / mm : INFINITY);
            if (dm == 0.0 || dm <= o.tol_scat * mm) break;
            if (it_adj >= o.max_it_scat) { conv_adj = false; break; }
            if (pbc) kl = 1 - kl;
        }
        CKL(launch_grad_scat(prec, Ifwd, lbuf[kl], N, G, nb, d0, c->w64, c->mesh.vol, d_dlg,
                            coupled ? c->J : nullptr, gk, ge, b_gks.p, c->st),
           "gradient");
    }
    cudaMemcpyKind kout = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(gk_out, gk, sizeof(double) * NG, kout, c->st), "copy gradient");
    CK(cudaMemcpyAsync(ge_out, ge, sizeof(double) * NG, kout, c->st), "copy gradient");
    if (gks_out) CK(cudaMemcpyAsync(gks_out, b_gks.p, sizeof(double) * NG, kout, c->st), "copy gradient");
    cudaEventRecord(t1, c->st);
    CK(cudaStreamSynchronize(c->st), "adjoint");
    float ttot = 0;
    cudaEventElapsedTime(&ttot, t0, t1);
    S.n_sweeps = n_sweeps;
    S.it_scat = it_fwd;
    S.it_pbc = it_adj;
    S.res_scat = res_fwd;
    S.res_pbc = res_adj;
    S.t_ms[0] = tcl;
    S.t_ms[1] = tlv;
    S.t_ms[2] = t_sweep;
    S.t_ms[4] = ttot;
    S.t_ms[5] = tasm;  // forward and transposed operators
    S.t_ms[6] = t_tr;  // the transposed sweeps alone
    S.updates = (double)N * D * G * (it_fwd + 2.0 * it_adj);  // forward, transposed over 2G split groups
    {
        const Levels& Ld = B == D ? c->lev : c->adj_lev;  // depths of the (last) batch levelised
        int dmaxv = 0;
        double dsum = 0;
        for (int d : Ld.depth) {
            dmaxv = std::max(dmaxv, d);
            dsum += d;
        }
        S.depth_max = dmaxv;
        S.depth_mean = Ld.depth.empty() ? 0.0 : dsum / Ld.depth.size();
    }
    S.updates_per_s = ttot > 0 ? S.updates / (ttot * 1e-3) : 0.0;
    S.schedule_used = plain ? SWEEP_SCHED_PLAIN : sched;
    S.kernel_used = c->last_kernel;
    S.kernel_launches = (int32_t)(c->launches - launches0);
    if (stats) *stats = S;
    return (conv_fwd && conv_adj) ? SWEEP_OK : SWEEP_NOT_CONVERGED;
}

}  // namespace

extern "C" {

sweep_status sweep_solve(sweep_ctx* c, const sweep_opts* o, double* J, double* Gam, sweep_stats* st) {
    return solve_impl(c, o, J, Gam, false, st);
}

sweep_status sweep_solve_dev(sweep_ctx* c, const sweep_opts* o, double* J, double* Gam, sweep_stats* st) {
    return solve_impl(c, o, J, Gam, true, st);
}

sweep_status sweep_levels(sweep_ctx* c, int32_t dir, int32_t* level, int32_t* depth) {
    if (!c) return SWEEP_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (!c->has_mesh || !c->has_dirs) return bad(c, "set mesh and directions first");
    if (dir < 0 || dir >= c->D) return bad(c, "direction index out of range");
    sweep_status s = ensure_levels(c, nullptr, nullptr, nullptr);
    if (s != SWEEP_OK) return s;
    if (level)
        CK(cudaMemcpyAsync(level, c->lev.level + (size_t)dir * c->mesh.N, sizeof(int32_t) * c->mesh.N,
                           cudaMemcpyDeviceToHost, c->st), "copy levels");
    CK(cudaStreamSynchronize(c->st), "copy levels");
    if (depth) *depth = c->lev.depth[dir];
    return SWEEP_OK;
}

sweep_status sweep_intensity(sweep_ctx* c, int32_t dir, double* out) {
    if (!c) return SWEEP_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (c->sb.last < 0 || !c->sb.I[c->sb.last]) return bad(c, "no solve yet");
    if (dir < 0 || dir >= c->sb.nd) return bad(c, "direction index out of range");
    if (!out) return bad(c, "null output");
    const size_t n = (size_t)c->sb.N * c->sb.G;
    double* tmp = nullptr;
    CK(cudaMalloc(&tmp, sizeof(double) * (n > 0 ? n : 1)), "alloc");
    const size_t es = c->sb.prec == 64 ? 8 : 4;
    const char* src = (const char*)c->sb.I[c->sb.last] + es * n * dir;
    cudaError_t e = launch_to_f64(c->sb.prec, src, (int64_t)n, tmp, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, sizeof(double) * n, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    cudaFree(tmp);
    return cuda_status(c, e, "copy intensity");
}

// Rotation of the direction set between substeps (Sec. 2.6, the rotation paragraph), with the remap of the
// intensities the last solve left (the warm start of the next periodic iteration).
sweep_status sweep_rotate_directions(sweep_ctx* c, const double* R, int64_t n_quad) {
    if (!c) return SWEEP_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (!c->has_dirs) return bad(c, "set the directions first");
    if (!R) return bad(c, "null rotation");
    if (n_quad == 0) n_quad = 1 << 16;
    if (n_quad < 1 || n_quad > (1ll << 26)) return bad(c, "n_quad must be in [1, 2^26] (0 = 2^16)");
    // a proper rotation: R^T R = 1 and det R = +1, within 1e-12
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += R[3 * k + a] * R[3 * k + b];
            if (!(std::fabs(s - (a == b ? 1.0 : 0.0)) <= 1e-12)) return bad(c, "rotation is not orthonormal");
        }
    const double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) +
                       R[2] * (R[3] * R[7] - R[4] * R[6]);
    if (!(std::fabs(det - 1.0) <= 1e-12)) return bad(c, "rotation must have determinant +1");
    const int D = c->D;
    std::vector<double> om_old(3 * (size_t)D), om_new(3 * (size_t)D), w(D);
    CK(cudaMemcpy(om_old.data(), c->om64, sizeof(double) * 3 * D, cudaMemcpyDeviceToHost), "read directions");
    CK(cudaMemcpy(w.data(), c->w64, sizeof(double) * D, cudaMemcpyDeviceToHost), "read directions");
    for (int d = 0; d < D; ++d)
        for (int k = 0; k < 3; ++k) {
            // ((R_k0 x + R_k1 y) + R_k2 z), each product and sum rounded on its own
            volatile double p0 = R[3 * k] * om_old[3 * d], p1 = R[3 * k + 1] * om_old[3 * d + 1],
                            p2 = R[3 * k + 2] * om_old[3 * d + 2];
            om_new[3 * d + k] = (p0 + p1) + p2;
        }
    SolveBuf& b = c->sb;
    const bool remap = b.last >= 0 && b.I[b.last] && b.nd == D;
    if (remap) {
        // quadrature points z_m = 1 - (2m+1)/M, phi_m = m pi (3 - sqrt 5) on the unit sphere
        std::vector<double3> pts((size_t)n_quad);
        const double golden = M_PI * (3.0 - std::sqrt(5.0));
        for (int64_t m = 0; m < n_quad; ++m) {
            const double z = 1.0 - (2.0 * (double)m + 1.0) / (double)n_quad;
            volatile double zz = z * z;
            const double r = std::sqrt(1.0 - zz);
            const double ph = (double)m * golden;
            pts[(size_t)m] = make_double3(r * std::cos(ph), r * std::sin(ph), z);
        }
        DevBuf<double3> d_pts;
        DevBuf<double> d_new;
        DevBuf<unsigned long long> d_cnt;
        CK(cudaMalloc(&d_pts.p, sizeof(double3) * (size_t)n_quad), "alloc quadrature");
        CK(cudaMalloc(&d_new.p, sizeof(double) * 3 * D), "alloc directions");
        CK(cudaMalloc(&d_cnt.p, sizeof(unsigned long long) * (size_t)D * D), "alloc counts");
        CK(cudaMemcpyAsync(d_pts.p, pts.data(), sizeof(double3) * (size_t)n_quad, cudaMemcpyHostToDevice, c->st),
           "upload");
        CK(cudaMemcpyAsync(d_new.p, om_new.data(), sizeof(double) * 3 * D, cudaMemcpyHostToDevice, c->st), "upload");
        CK(cudaMemsetAsync(d_cnt.p, 0, sizeof(unsigned long long) * (size_t)D * D, c->st), "init");
        CKL(launch_remap_count(d_pts.p, n_quad, c->om64, d_new.p, D, d_cnt.p, c->st), "remap coefficients");
        std::vector<unsigned long long> cnt((size_t)D * D);
        CK(cudaMemcpyAsync(cnt.data(), d_cnt.p, sizeof(unsigned long long) * (size_t)D * D, cudaMemcpyDeviceToHost,
                           c->st), "read counts");
        CK(cudaStreamSynchronize(c->st), "remap coefficients");
        // c_ij = dS_ij / dS_i as a sparse matrix by rows (new directions)
        std::vector<int32_t> rp(D + 1, 0), col;
        std::vector<double> val;
        for (int i = 0; i < D; ++i) {
            unsigned long long row = 0;
            for (int j = 0; j < D; ++j) row += cnt[(size_t)i * D + j];
            for (int j = 0; j < D; ++j) {
                const unsigned long long n = cnt[(size_t)i * D + j];
                if (!n) continue;
                col.push_back(j);
                val.push_back((double)n / (double)row);
            }
            rp[i + 1] = (int32_t)col.size();
        }
        DevBuf<int32_t> d_rp, d_col;
        DevBuf<double> d_val;
        const size_t nnz = col.size() > 0 ? col.size() : 1;
        CK(cudaMalloc(&d_rp.p, sizeof(int32_t) * (D + 1)), "alloc remap");
        CK(cudaMalloc(&d_col.p, sizeof(int32_t) * nnz), "alloc remap");
        CK(cudaMalloc(&d_val.p, sizeof(double) * nnz), "alloc remap");
        CK(cudaMemcpyAsync(d_rp.p, rp.data(), sizeof(int32_t) * (D + 1), cudaMemcpyHostToDevice, c->st), "upload");
        CK(cudaMemcpyAsync(d_col.p, col.data(), sizeof(int32_t) * col.size(), cudaMemcpyHostToDevice, c->st), "upload");
        CK(cudaMemcpyAsync(d_val.p, val.data(), sizeof(double) * val.size(), cudaMemcpyHostToDevice, c->st), "upload");
        // remap the last solve's intensities into the other buffer, which becomes the last one
        const int src = b.last, dst = 1 - b.last;
        if (!b.I[dst]) {
            CK(cudaMalloc(&b.I[dst], b.bytes > 0 ? b.bytes : 4), "alloc intensities");
            b.sign[dst] = 0;
        }
        const int64_t NG = b.N * (int64_t)b.G;
        CKL(launch_remap(b.prec, b.I[src], b.I[dst], NG, D, d_rp.p, d_col.p, d_val.p, b.sign[dst], c->st), "remap");
        CK(cudaStreamSynchronize(c->st), "remap");
        b.last = dst;
    }
    // the rotated set replaces the directions (weights unchanged); levels and operators are rebuilt
    std::vector<float4> o32(D), o32lo(D);
    for (int d = 0; d < D; ++d) {
        const double* x = om_new.data() + 3 * d;
        o32[d] = make_float4((float)x[0], (float)x[1], (float)x[2], (float)w[d]);
        o32lo[d] = make_float4((float)(x[0] - (double)o32[d].x), (float)(x[1] - (double)o32[d].y),
                               (float)(x[2] - (double)o32[d].z), 0.f);
    }
    CK(cudaMemcpy(c->om64, om_new.data(), sizeof(double) * 3 * D, cudaMemcpyHostToDevice), "upload directions");
    CK(cudaMemcpy(c->om32, o32.data(), sizeof(float4) * D, cudaMemcpyHostToDevice), "upload directions");
    CK(cudaMemcpy(c->om32lo, o32lo.data(), sizeof(float4) * D, cudaMemcpyHostToDevice), "upload directions");
    c->lev.valid = false;
    c->lev.op_valid = false;
    c->lev.pkt.valid = false;
    c->adj_lev.valid = false;
    return SWEEP_OK;
}

sweep_status sweep_adjoint(sweep_ctx* c, const sweep_opts* o, const double* dlj, const double* dlg, double* gk,
                           double* ge, double* gks, sweep_stats* st) {
    return adjoint_impl(c, o, dlj, dlg, gk, ge, gks, false, st);
}

sweep_status sweep_adjoint_dev(sweep_ctx* c, const sweep_opts* o, const double* dlj, const double* dlg, double* gk,
                               double* ge, double* gks, sweep_stats* st) {
    return adjoint_impl(c, o, dlj, dlg, gk, ge, gks, true, st);
}

}  // extern "C"
