// The transport sweep (K3 batched, K8 plain) and its transpose (adjoint).
//
// Cell update -- transport scheme (a) of paper Sec. 2.6: the total outflow F of a task (c, Omega)
// leaves through downwind face i in proportion to A_i (n_i.Omega). As a balance over the cell,
//     (P_c + kappa_t,c V_c) I_c = q_c + sum_{inflow sides} |a_f| I_up(f),   a_f = A_f n_f.Omega,
// with P_c the projected outflow area (sum of a_f over outflow sides, boundary and periodic
// included) and q_c = eps_c/(4 pi) + kappa_s,c V_c J_c the emission plus the scattering source
// of Alg. 1. Inflow from a periodic side is the partner cell's intensity of the previous
// periodic iteration (Sec. 2.7); inflow from a boundary side is the boundary intensity (vacuum: 0).
//
// The adjoint solves L^T lambda = g per direction: lambda_c = (g_c + sum_{outflow interior sides}
// |a_f| lambda_down(f)) / (P_c + kappa_t,c V_c), i.e. the same row data swept in reversed level order.
//
// Schedules (all directions and all meshes of a batch in one persistent launch):
//   LEVEL    -- warps take chunks (32/L tasks, L lanes each) of one wavefront level round-robin;
//               grid barrier per level.
//   DATAFLOW -- no barriers: warp w takes chunks w, w+W, ... in level order and each task waits
//               (bounded) until its upwind values are written. Every dependency sits in an earlier
//               level, hence an earlier chunk, so the lowest unfinished chunk can always progress.
// Readiness is carried by the value itself: every sweep writes its intensities with a sign bit equal
// to the sweep's parity (values are >= 0), so a reader knows whether it sees this sweep's value.
#include "common.cuh"

namespace sw {
namespace {

template <typename real> struct vec2;
template <> struct vec2<float> { using type = float2; };
template <> struct vec2<double> { using type = double2; };

__device__ __forceinline__ float addr(float a, float b) { return a + b; }
__device__ __forceinline__ double addr(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mulr(float a, float b) { return a * b; }
__device__ __forceinline__ double mulr(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fmar(float a, float b, float c) { return fmaf(a, b, c); }
// FP64 path: separately rounded multiply and add, the oracle's rounding sequence
__device__ __forceinline__ double fmar(double a, double b, double c) { return __dadd_rn(c, __dmul_rn(a, b)); }
// FP32 path: fast division (relative error ~2 ulp, far inside the FP32 tolerance); denominators are
// projected areas plus kappa*V, never near the 2^126 range where the fast form underflows
__device__ __forceinline__ float divr(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double divr(double a, double b) { return __ddiv_rn(a, b); }

// EXP law of one cell and group: outgoing (exp(-tau) F_in + q) / P and cell mean (F_in / P)(1 - exp(-tau)) / tau,
// tau = kappa_t V / P; with no outflow (P = 0) everything that enters or is emitted stays: (q + F_in) / kappa_t V
__device__ __forceinline__ void exp_update(float fin, float q, float ktv, float P, float& out, float& mean) {
    if (P > 0.f) {
        const float tau = ktv / P;
        const float f = tau > 0.f ? -expm1f(-tau) / tau : 1.f;
        out = fmaf(expf(-tau), fin, q) / P;
        mean = fin / P * f;
    } else {
        out = mean = (q + fin) / ktv;
    }
}
__device__ __forceinline__ void exp_update(double fin, double q, double ktv, double P, double& out, double& mean) {
    if (P > 0.0) {
        const double tau = ktv / P;
        const double f = tau > 0.0 ? -expm1(-tau) / tau : 1.0;
        out = (exp(-tau) * fin + q) / P;
        mean = fin / P * f;
    } else {
        out = mean = (q + fin) / ktv;
    }
}
// The same law in the packed kernel, where every lane of a packet evaluates it (the head lanes keep the
// result): one expf and two fast reciprocals, selects instead of branches. The mean factor
// f = (1 - exp(-tau)) / tau is taken from its Taylor series sum_k (-tau)^k / (k+1)! (seven terms,
// truncation below 2e-9) where 1 - exp(-tau) would cancel (tau < 1/4), and directly above.
__device__ __forceinline__ void exp_update_lanes(float fin, float q, float ktv, float P, float& out, float& mean) {
    const float rP = __fdividef(1.f, P), rK = __fdividef(1.f, ktv);
    const float tau = ktv * rP;
    const float e = expf(-tau);
    const float s = -tau;
    float ft = fmaf(s, 1.f / 5040.f, 1.f / 720.f);
    ft = fmaf(s, ft, 1.f / 120.f);
    ft = fmaf(s, ft, 1.f / 24.f);
    ft = fmaf(s, ft, 1.f / 6.f);
    ft = fmaf(s, ft, 0.5f);
    ft = fmaf(s, ft, 1.f);
    const float f = tau < 0.25f ? ft : (1.f - e) * P * rK;
    const float stay = (q + fin) * rK;  // P = 0: no outflow
    out = P > 0.f ? fmaf(e, fin, q) * rP : stay;
    mean = P > 0.f ? fin * rP * f : stay;
}
// out of line in the mesh-row kernels, whose common path stays short
__device__ __noinline__ void exp_law(float fin, float q, float ktv, float P, float& out, float& mean) {
    exp_update(fin, q, ktv, P, out, mean);
}
__device__ __noinline__ void exp_law(double fin, double q, double ktv, double P, double& out, double& mean) {
    exp_update(fin, q, ktv, P, out, mean);
}

// Rare path, kept out of line so the common path stays short:
// Wait (bounded) until *p carries this sweep's parity; returns the magnitude. false on give-up.
template <typename real>
__device__ __noinline__ bool wait_value_slow(const real* p, int parity, const SweepArgs& a, real& out);

template <typename real>
__device__ __forceinline__ bool wait_value(const real* p, int parity, const SweepArgs& a, real& out) {
    real v = ld_relaxed(p);
    if (sign_bit(v) == (parity != 0)) {
        out = parity ? -v : v;
        return true;
    }
    long long n = 0;
    for (;;) {
        ++n;
        if (n > a.spin_budget || ((n & 63) == 0 && ld_volatile_i32(a.err) != DEV_OK)) {
            atomicCAS(a.err, DEV_OK, DEV_TIMEOUT);
            return false;
        }
        __nanosleep(20);
        v = ld_relaxed(p);
        if (sign_bit(v) == (parity != 0)) {
            out = parity ? -v : v;
            return true;
        }
    }
}

template <typename real>
__device__ __noinline__ bool wait_value_slow(const real* p, int parity, const SweepArgs& a, real& out) {
    return wait_value(p, parity, a, out);
}

// ---------------------------------------------------------------------------------------------
// Batched sweep: L lanes cooperate on one task (c, Omega). Each lane owns the face sides
// r0 + lane + k*L (k < U = SLOTS/L), so one pass covers SLOTS = 16 sides (a Voronoi cell has 15.5
// on average) with coalesced 16-byte record loads that are all in flight together; the upwind
// reads of the pass are issued together too; P_c and the inflow sums are reduced over the L lanes
// with shuffles.
// ---------------------------------------------------------------------------------------------
constexpr int SLOTS = 16;
// L2 prefetch of a task's face-side row by the bulk-copy engine (the row is contiguous, 16-byte
// records, so address and size are multiples of 16 bytes)
__device__ __forceinline__ void prefetch_row(const int4* side, uint32_t r0, uint32_t r1) {
    if (r1 > r0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(side + r0), "r"((r1 - r0) * 16u));
}

template <typename real, int GC, int L>
__device__ __forceinline__ bool group_task(const SweepArgs& a, uint32_t entry, uint32_t r0, uint32_t r1,
                                           const float4* s_om, int gl, bool stall, uint64_t pol) {
    constexpr bool F64 = sizeof(real) == 8;
    constexpr int GM = GC > 0 ? GC : 8;
    constexpr int U = L == 1 ? 8 : SLOTS / L;  // face sides per lane per pass
    constexpr int PASS = L * U;                 // face sides per pass
    const int G = GC > 0 ? GC : a.G;
    using real2 = typename vec2<real>::type;
    const bool valid = entry != TASK_PAD;
    const uint32_t c = valid ? (entry & a.cmask) : 0u;
    const uint32_t dl = valid ? (entry >> a.cshift) : 0u;
    if (!valid) r1 = r0;
    // source and denominator of the cell, loaded early (used after the reduction)
    real2 q[GM];
    if (valid && gl == 0) {
        const real2* cm = reinterpret_cast<const real2*>(a.cm) + (size_t)c * G;
#pragma unroll
        for (int g = 0; g < GM; ++g)
            if (g < G) q[g] = cm[g];
    }
    const double* om64 = a.om64 + 3 * dl;
    const float4 om = s_om[dl];
    const float4 oml = F64 ? make_float4(0.f, 0.f, 0.f, 0.f) : a.om32lo[dl];
    real* I = reinterpret_cast<real*>(a.I);
    const size_t slab = (size_t)dl * a.N;
    bool fail = false;
    if (stall && gl == 0) {  // test hook: wait on a word that nothing writes
        real dummy;
        if (!wait_value(reinterpret_cast<const real*>(a.stall_word), 1, a, dummy)) fail = true;
    }
    real P = 0;
    real acc[GM];
#pragma unroll
    for (int g = 0; g < GM; ++g) acc[g] = 0;
    for (uint32_t base = r0; base < r1; base += PASS) {
        int4 rec[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t s = base + gl + k * L;
            rec[k] = s < r1 ? ld_stream_int4(a.side + s, pol) : make_int4(0, 0, 0, 0);
        }
        real w[U];
        int kind[U];  // 0 none, 1 interior inflow, 2 periodic inflow (adjoint: its transpose), 3 boundary inflow
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t s = base + gl + k * L;
            kind[k] = 0;
            w[k] = 0;
            if (s < r1) {
                int sgn;
                if (F64) {
                    const d4 n = a.side64[s];
                    const double t = exact_t(n, om64);
                    sgn = t > 0.0 ? 1 : (t < 0.0 ? -1 : 0);
                    w[k] = (real)__dmul_rn(n.w, fabs(t));
                } else {
                    const float ax = __int_as_float(rec[k].y), ay = __int_as_float(rec[k].z),
                                az = __int_as_float(rec[k].w);
                    sgn = classify_side(dot32(ax, ay, az, om), ax, ay, az, a.side64, s, om64);
                    if (sgn != 0) w[k] = (real)side_weight(rec[k], a.side_lo[s], om, oml);
                }
                if (sgn > 0) P = addr(P, w[k]);
                const bool inflow = sgn != 0 && (a.reverse ? (sgn > 0) : (sgn < 0));
                if (inflow) {
                    const int32_t nb = rec[k].x;
                    if (nb >= 0 && !(nb & NBR_PERIODIC)) kind[k] = 1;
                    else if (nb >= 0) kind[k] = 2;  // the partner's value of the previous sweep or pass
                    else if (!a.reverse) kind[k] = 3;
                    if (a.dc_mask && nb >= 0) {  // scheme (b): the upwind cell's share, if it chose this face
                        const int64_t i = (int64_t)(nb & NBR_MASK) * a.nd + dl;
                        if ((a.dc_mask[i] >> a.twin[s]) & 1ull) w[k] = F64 ? (real)a.dc_share64[i] : (real)a.dc_share32[i];
                        else kind[k] = 0;
                    }
                }
            }
        }
        // upwind reads of the pass, all issued before any is used
        real v[U][GM];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            if (kind[k] == 1) {
                const real* src = I + (slab + (uint32_t)rec[k].x) * G;
#pragma unroll
                for (int g = 0; g < GM; ++g)
                    if (g < G) v[k][g] = ld_relaxed(src + g);
            }
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            if (kind[k] == 1) {
                const real* src = I + (slab + (uint32_t)rec[k].x) * G;
#pragma unroll
                for (int g = 0; g < GM; ++g) {
                    if (g < G) {
                        real x = v[k][g];
                        if (sign_bit(x) != (a.parity != 0)) {
                            if (fail || !wait_value_slow(src + g, a.parity, a, x)) {
                                fail = true;
                                x = 0;
                            }
                        } else {
                            x = a.parity ? -x : x;
                        }
                        acc[g] = fmar(w[k], x, acc[g]);
                    }
                }
            } else if (kind[k] == 2) {
                if (a.Iprev) {
                    const real* src = reinterpret_cast<const real*>(a.Iprev) +
                                      (slab + (uint32_t)(rec[k].x & NBR_MASK)) * G;
#pragma unroll
                    for (int g = 0; g < GM; ++g)
                        if (g < G) acc[g] = fmar(w[k], (real)fabs(src[g]), acc[g]);
                }
            } else if (kind[k] == 3) {
                if (a.bc) {
                    const real* b = reinterpret_cast<const real*>(a.bc) + (size_t)(-1 - rec[k].x) * G;
#pragma unroll
                    for (int g = 0; g < GM; ++g)
                        if (g < G) acc[g] = fmar(w[k], b[g], acc[g]);
                }
            }
        }
    }
    // reduce over the L lanes of the group (aligned sub-warp, xor offsets stay inside it)
#pragma unroll
    for (int off = L / 2; off > 0; off >>= 1) {
        P = addr(P, __shfl_xor_sync(0xffffffffu, P, off));
#pragma unroll
        for (int g = 0; g < GM; ++g)
            if (g < G) acc[g] = addr(acc[g], __shfl_xor_sync(0xffffffffu, acc[g], off));
    }
    if (valid && gl == 0 && !fail) {
        const real wsc = a.reverse ? (real)a.w64[dl] : (real)1;
        real* dst = I + (slab + c) * G;
#pragma unroll
        for (int g = 0; g < GM; ++g) {
            if (g < G) {
                if (a.law) {
                    real val, mean;
                    exp_law(acc[g], q[g].x, q[g].y, P, val, mean);
                    reinterpret_cast<real*>(a.Imean)[(slab + c) * G + g] = mean;
                    st_relaxed(dst + g, a.parity ? -val : val);
                    continue;
                }
                const real src = a.reverse ? mulr(wsc, q[g].x) : q[g].x;
                const real val = divr(addr(src, acc[g]), addr(P, q[g].y));
                st_relaxed(dst + g, a.parity ? -val : val);
            }
        }
    }
    return !fail;
}

// row bounds of a task entry (0, 0 for padding)
__device__ __forceinline__ uint2 row_of(const SweepArgs& a, uint32_t e) {
    if (e == TASK_PAD) return make_uint2(0u, 0u);
    const uint32_t c = e & a.cmask;
    return make_uint2(__ldg(a.rowptr + c), __ldg(a.rowptr + c + 1));
}

// A warp walks its chunks (32/L tasks, one per lane group) in order. Software pipeline: task entries
// are loaded PF+1 chunks ahead, row bounds PF chunks ahead, and the face-side rows PF-1 chunks ahead
// are pulled into L2 by the bulk-copy engine, so a task's records are L2 hits when it runs.
// chunk(i) gives the i-th chunk of this warp, or -1 past the end.
template <typename real, int GC, int L, typename ChunkFn>
__device__ __forceinline__ bool run_chunks(const SweepArgs& a, ChunkFn chunk, const float4* s_om, int grp, int gl,
                                           bool stall_here) {
    const uint64_t pol = policy_evict_first();
    constexpr int CS = 32 / L;
    constexpr int PF = 3;
    auto entry_of = [&](int64_t i) -> uint32_t {
        const int64_t k = chunk(i);
        return k >= 0 ? a.task[k * CS + grp] : TASK_PAD;
    };
    uint32_t E[PF + 1];
    uint2 R[PF];
#pragma unroll
    for (int j = 0; j <= PF; ++j) E[j] = entry_of(j);
#pragma unroll
    for (int j = 0; j < PF; ++j) R[j] = row_of(a, E[j]);
    if (gl == 0) {
#pragma unroll
        for (int j = 1; j < PF - 1; ++j) prefetch_row(a.side, R[j].x, R[j].y);
    }
    for (int64_t i = 0; chunk(i) >= 0; ++i) {
        if ((i & 15) == 0 && __any_sync(0xffffffffu, ld_volatile_i32(a.err) != DEV_OK)) return false;
        const uint32_t e_new = entry_of(i + PF + 1);
        const uint2 r_new = row_of(a, E[PF]);
        if (gl == 0) prefetch_row(a.side, R[PF - 1].x, R[PF - 1].y);
        const bool stall = stall_here && i == 0 && grp == 0;
        const bool good = group_task<real, GC, L>(a, E[0], R[0].x, R[0].y, s_om, gl, stall, pol);
        if (__any_sync(0xffffffffu, !good)) return false;
#pragma unroll
        for (int j = 0; j < PF; ++j) E[j] = E[j + 1];
        E[PF] = e_new;
#pragma unroll
        for (int j = 0; j < PF - 1; ++j) R[j] = R[j + 1];
        R[PF - 1] = r_new;
    }
    return true;
}

// ---------------------------------------------------------------------------------------------
// FP32 forward sweep from task records. The classification pass already fixed, per task, P_c and
// which of the first 32 face sides are inflow sides, so a task only visits its inflow sides
// (about half the row): no classification, no outflow sum. L lanes share a task, lane j taking
// the inflow sides of rank j, j+L, ...; each batch issues U record loads, then U upwind loads.
// Rows longer than 32 sides (rare) classify their remaining sides on the spot.
// ---------------------------------------------------------------------------------------------
template <int GC>
__device__ __forceinline__ void add_inflow(const SweepArgs& a, int32_t nb, float w, const float* vpre, size_t slab,
                                           int G, float* acc, bool& fail) {
    constexpr int GM = GC > 0 ? GC : 8;
    if (nb >= 0 && !(nb & NBR_PERIODIC)) {
        const float* src = reinterpret_cast<const float*>(a.I) + (slab + (uint32_t)nb) * G;
#pragma unroll
        for (int g = 0; g < GM; ++g) {
            if (g < G) {
                float x = vpre ? vpre[g] : ld_relaxed(src + g);
                if (sign_bit(x) != (a.parity != 0)) {
                    if (fail || !wait_value_slow(src + g, a.parity, a, x)) {
                        fail = true;
                        x = 0.f;
                    }
                } else {
                    x = a.parity ? -x : x;
                }
                acc[g] = fmaf(w, x, acc[g]);
            }
        }
    } else if (nb >= 0) {
        if (a.Iprev) {
            const float* src = reinterpret_cast<const float*>(a.Iprev) + (slab + (uint32_t)(nb & NBR_MASK)) * G;
#pragma unroll
            for (int g = 0; g < GM; ++g)
                if (g < G) acc[g] = fmaf(w, fabsf(src[g]), acc[g]);
        }
    } else if (a.bc) {
        const float* b = reinterpret_cast<const float*>(a.bc) + (size_t)(-1 - nb) * G;
#pragma unroll
        for (int g = 0; g < GM; ++g)
            if (g < G) acc[g] = fmaf(w, b[g], acc[g]);
    }
}

template <int GC, int L>
__device__ __forceinline__ bool rec_task(const SweepArgs& a, const int4 tr, const float4* s_om, int gl, bool stall,
                                         uint64_t pol) {
    constexpr int GM = GC > 0 ? GC : 8;
    constexpr int U = 8 / L;  // inflow sides per lane per batch
    const int G = GC > 0 ? GC : a.G;
    const uint32_t e = (uint32_t)tr.x;
    const bool valid = e != TASK_PAD;
    const uint32_t c = valid ? (e & a.cmask) : 0u;
    const uint32_t dl = valid ? (e >> a.cshift) : 0u;
    const uint32_t r0 = (uint32_t)tr.y;
    const float P = __int_as_float(tr.z & 0x7fffffff);
    const bool longrow = valid && tr.z < 0;
    uint32_t m = valid ? (uint32_t)tr.w : 0u;
#pragma unroll
    for (int j = 0; j < L - 1; ++j)
        if (j < gl) m &= m - 1;  // this lane starts at the inflow side of rank gl
    float2 q[GM];
    if (valid && gl == 0) {
        const float2* cm = reinterpret_cast<const float2*>(a.cm) + (size_t)c * G;
#pragma unroll
        for (int g = 0; g < GM; ++g)
            if (g < G) q[g] = cm[g];
    }
    const float4 om = s_om[dl];
    const float4 oml = a.om32lo[valid ? dl : 0u];
    const size_t slab = (size_t)dl * a.N;
    bool fail = false;
    if (stall && gl == 0) {
        float dummy;
        if (!wait_value(reinterpret_cast<const float*>(a.stall_word), 1, a, dummy)) fail = true;
    }
    float acc[GM];
#pragma unroll
    for (int g = 0; g < GM; ++g) acc[g] = 0.f;
    while (m) {
        uint32_t pos[U];
        bool ok[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            ok[k] = m != 0u;
            pos[k] = ok[k] ? (uint32_t)(__ffs(m) - 1) : 0u;
#pragma unroll
            for (int j = 0; j < L; ++j) m &= m - 1;
        }
        int4 rec[U];
#pragma unroll
        for (int k = 0; k < U; ++k) rec[k] = ok[k] ? ld_stream_int4(a.side + r0 + pos[k], pol) : make_int4(-1, 0, 0, 0);
        float v[U][GM];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            if (ok[k] && rec[k].x >= 0 && !(rec[k].x & NBR_PERIODIC)) {
                const float* src = reinterpret_cast<const float*>(a.I) + (slab + (uint32_t)rec[k].x) * G;
#pragma unroll
                for (int g = 0; g < GM; ++g)
                    if (g < G) v[k][g] = ld_relaxed(src + g);
            }
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            if (!ok[k]) continue;
            const float w = side_weight(rec[k], __ldg(a.side_lo + r0 + pos[k]), om, oml);
            add_inflow<GC>(a, rec[k].x, w, v[k], slab, G, acc, fail);
        }
    }
    if (longrow) {
        const uint32_t r1 = __ldg(a.rowptr + c + 1);
        const double* om64 = a.om64 + 3 * dl;
        for (uint32_t s = r0 + 32 + gl; s < r1; s += L) {
            const int4 r = a.side[s];
            const float ax = __int_as_float(r.y), ay = __int_as_float(r.z), az = __int_as_float(r.w);
            if (classify_side(dot32(ax, ay, az, om), ax, ay, az, a.side64, s, om64) < 0)
                add_inflow<GC>(a, r.x, side_weight(r, a.side_lo[s], om, oml), nullptr, slab, G, acc, fail);
        }
    }
#pragma unroll
    for (int off = L / 2; off > 0; off >>= 1) {
#pragma unroll
        for (int g = 0; g < GM; ++g)
            if (g < G) acc[g] += __shfl_xor_sync(0xffffffffu, acc[g], off);
    }
    if (valid && gl == 0 && !fail) {
        float* dst = reinterpret_cast<float*>(a.I) + (slab + c) * G;
#pragma unroll
        for (int g = 0; g < GM; ++g) {
            if (g < G) {
                const float val = __fdividef(q[g].x + acc[g], P + q[g].y);
                st_relaxed(dst + g, a.parity ? -val : val);
            }
        }
    }
    return !fail;
}

// the highest inflow side bounds the part of the row a record's task reads
__device__ __forceinline__ void prefetch_rec(const SweepArgs& a, const int4 tr) {
    if ((uint32_t)tr.x == TASK_PAD || tr.w == 0) return;
    const uint32_t n = 32u - __clz((uint32_t)tr.w);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.side + (uint32_t)tr.y), "r"(n * 16u));
}

template <int GC, int L, typename ChunkFn>
__device__ __forceinline__ bool run_chunks_rec(const SweepArgs& a, ChunkFn chunk, const float4* s_om, int grp, int gl,
                                               bool stall_here) {
    constexpr int CS = 32 / L;
    constexpr int PF = 3;
    const uint64_t pol = policy_evict_first();
    auto rec_of = [&](int64_t i) -> int4 {
        const int64_t k = chunk(i);
        return k >= 0 ? __ldg(a.trec + k * CS + grp) : make_int4((int)TASK_PAD, 0, 0, 0);
    };
    int4 T[PF + 1];
#pragma unroll
    for (int j = 0; j <= PF; ++j) T[j] = rec_of(j);
    if (gl == 0) {
#pragma unroll
        for (int j = 1; j < PF; ++j) prefetch_rec(a, T[j]);
    }
    for (int64_t i = 0; chunk(i) >= 0; ++i) {
        if ((i & 15) == 0 && __any_sync(0xffffffffu, ld_volatile_i32(a.err) != DEV_OK)) return false;
        const int4 t_new = rec_of(i + PF + 1);
        if (gl == 0) prefetch_rec(a, T[PF]);
        const bool stall = stall_here && i == 0 && grp == 0;
        const bool good = rec_task<GC, L>(a, T[0], s_om, gl, stall, pol);
        if (__any_sync(0xffffffffu, !good)) return false;
#pragma unroll
        for (int j = 0; j < PF; ++j) T[j] = T[j + 1];
        T[PF] = t_new;
    }
    return true;
}

template <int GC, int L>
#ifndef SWEEP_REC_MINB
#define SWEEP_REC_MINB 4  // resident 256-thread blocks per SM the record kernel is compiled for
#endif
__global__ void __launch_bounds__(256, SWEEP_REC_MINB) k_sweep_rec(SweepArgs a) {
    extern __shared__ float4 s_om[];
    for (int i = threadIdx.x; i < a.nd; i += blockDim.x) s_om[i] = a.om32[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int grp = lane / L, gl = lane % L;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nchunks = a.n_chunks * L;
    if (a.level_sync) {
        bool ok = true;
        for (int li = 0; li < a.n_levels; ++li) {
            const int64_t k0 = a.lev_chunk[li] * L, k1 = a.lev_chunk[li + 1] * L;
            if (ok) {
                auto chunk = [=](int64_t i) -> int64_t {
                    const int64_t k = k0 + warp + i * nwarps;
                    return k < k1 ? k : -1;
                };
                ok = run_chunks_rec<GC, L>(a, chunk, s_om, grp, gl, a.debug_stall && li == 0 && warp == 0);
            }
            if (!grid_sync(a.bar, gridDim.x, a.spin_budget, a.err)) return;
        }
    } else {
        auto chunk = [=](int64_t i) -> int64_t {
            const int64_t k = warp + i * nwarps;
            return k < nchunks ? k : -1;
        };
        run_chunks_rec<GC, L>(a, chunk, s_om, grp, gl, a.debug_stall && warp == 0);
    }
}

template <typename real, int GC, int L>
__global__ void __launch_bounds__(256) k_sweep(SweepArgs a) {
    extern __shared__ float4 s_om[];
    for (int i = threadIdx.x; i < a.nd; i += blockDim.x) s_om[i] = a.om32[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int grp = lane / L, gl = lane % L;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nchunks = a.n_chunks * L;  // n_chunks counts 32-task chunks
    if (a.level_sync) {
        bool ok = true;
        for (int li = 0; li < a.n_levels; ++li) {
            const int Lv = a.reverse ? a.n_levels - 1 - li : li;
            const int64_t k0 = a.lev_chunk[Lv] * L, k1 = a.lev_chunk[Lv + 1] * L;
            if (ok) {
                auto chunk = [=](int64_t i) -> int64_t {
                    const int64_t k = k0 + warp + i * nwarps;
                    return k < k1 ? k : -1;
                };
                ok = run_chunks<real, GC, L>(a, chunk, s_om, grp, gl, a.debug_stall && li == 0 && warp == 0);
            }
            if (!grid_sync(a.bar, gridDim.x, a.spin_budget, a.err)) return;
        }
    } else {
        auto chunk = [=](int64_t i) -> int64_t {
            const int64_t k = a.reverse ? (nchunks - 1 - warp - i * nwarps) : (warp + i * nwarps);
            return (k >= 0 && k < nchunks) ? k : -1;
        };
        run_chunks<real, GC, L>(a, chunk, s_om, grp, gl, a.debug_stall && warp == 0);
    }
}

// ---------------------------------------------------------------------------------------------
// FP32 forward sweep over the assembled operator (one 128-byte line per task, see k_build_op). LP
// lanes share a task's line: lane j holds pieces [j*PL, (j+1)*PL) (PL = 8/LP pieces of 16 bytes;
// piece 0 is the header, piece p >= 1 holds entries 2p-2 and 2p-1), so one coalesced load brings
// the whole row of L_Omega; the upwind values are gathered, reduced over the LP lanes, and lane 0
// solves the cell.
// ---------------------------------------------------------------------------------------------
template <int LP>
struct OpPieces {
    int4 p[8 / LP];
};

// rows with more inflow sides than a line holds take the geometry path (kept out of line)
template <int GC, int LP>
__device__ __noinline__ bool op_overflow(const SweepArgs& a, int4 tr, const float4* s_om, int gl) {
    return rec_task<GC, LP>(a, tr, s_om, gl, false, policy_evict_first());
}

// an upwind value not yet written by this sweep: bounded wait (out of line, rare)
__device__ __noinline__ float op_wait(const SweepArgs& a, const float* p, bool& fail) {
    float x = 0.f;
    if (fail || !wait_value_slow(p, a.parity, a, x)) {
        fail = true;
        return 0.f;
    }
    return x;
}

// inflow through a periodic face (previous iteration's partner intensity) or a boundary face
template <int GC>
__device__ __forceinline__ void op_external(const SweepArgs& a, uint32_t idx, float w, bool boundary, int G,
                                            float* acc) {
    constexpr int GM = GC > 0 ? GC : 8;
    const float aw = -w;  // external entries carry the weight with its sign bit set
    if (boundary) {
        if (a.bc) {
            const float* b = reinterpret_cast<const float*>(a.bc) + (size_t)idx * G;
#pragma unroll
            for (int g = 0; g < GM; ++g)
                if (g < G) acc[g] = fmaf(aw, b[g], acc[g]);
        }
    } else if (a.Iprev) {
        const float* src = reinterpret_cast<const float*>(a.Iprev) + (size_t)idx * G;
#pragma unroll
        for (int g = 0; g < GM; ++g)
            if (g < G) acc[g] = fmaf(aw, fabsf(src[g]), acc[g]);
    }
}

template <int GC, int LP>
__device__ __forceinline__ bool op_task(const SweepArgs& a, const OpPieces<LP>& mine, int gl, bool stall,
                                        bool& overflow) {
    constexpr int GM = GC > 0 ? GC : 8;
    constexpr int PL = 8 / LP;
    const int G = GC > 0 ? GC : a.G;
    const int lead = (threadIdx.x & 31) & ~(LP - 1);
    const int4 h = mine.p[0];
    const uint32_t e = (uint32_t)__shfl_sync(0xffffffffu, h.x, lead);
    const float P = __int_as_float(__shfl_sync(0xffffffffu, h.y, lead));
    const int nz = __shfl_sync(0xffffffffu, h.z, lead);
    const uint32_t dst = (uint32_t)__shfl_sync(0xffffffffu, h.w, lead);
    const int nin = nz & 0xff;
    const bool valid = e != TASK_PAD;
    overflow = valid && nin > OP_MAX;
    const uint32_t c = valid ? (e & a.cmask) : 0u;
    const uint32_t par = a.parity ? 0x80000000u : 0u;
    float2 q[GM];
    if (valid && gl == 0 && !overflow) {
        const float2* cm = reinterpret_cast<const float2*>(a.cm) + (size_t)c * G;
#pragma unroll
        for (int g = 0; g < GM; ++g)
            if (g < G) q[g] = cm[g];
    }
    bool fail = false;
    if (stall && gl == 0) {
        float dummy;
        if (!wait_value(reinterpret_cast<const float*>(a.stall_word), 1, a, dummy)) fail = true;
    }
    float acc[GM];
#pragma unroll
    for (int g = 0; g < GM; ++g) acc[g] = 0.f;
    if (valid && !overflow) {
        constexpr int NE = 2 * PL;  // entry slots this lane holds
        uint32_t idx[NE];
        float w[NE];
        bool has[NE];
        int j[NE];
#pragma unroll
        for (int k = 0; k < PL; ++k) {
            const int piece = gl * PL + k;
            const int4 q4 = mine.p[k];
            j[2 * k] = 2 * piece - 2;
            j[2 * k + 1] = 2 * piece - 1;
            has[2 * k] = piece > 0 && j[2 * k] < nin;
            has[2 * k + 1] = piece > 0 && j[2 * k + 1] < nin;
            idx[2 * k] = (uint32_t)q4.x;
            w[2 * k] = __int_as_float(q4.y);
            idx[2 * k + 1] = (uint32_t)q4.z;
            w[2 * k + 1] = __int_as_float(q4.w);
        }
        float v[NE][GM];
        const float* I = reinterpret_cast<const float*>(a.I);
#pragma unroll
        for (int k = 0; k < NE; ++k) {  // issue every upwind read before using any
            if (has[k] && !sign_bit(w[k])) {
                const float* src = I + (size_t)idx[k] * G;
                if constexpr (GC == 4) {
                    const float4 q4 = ld_relaxed_v4(src);
                    v[k][0] = q4.x; v[k][1] = q4.y; v[k][2] = q4.z; v[k][3] = q4.w;
                } else if constexpr (GC == 2) {
                    const float2 q2 = ld_relaxed_v2(src);
                    v[k][0] = q2.x; v[k][1] = q2.y;
                } else {
#pragma unroll
                    for (int g = 0; g < GM; ++g)
                        if (g < G) v[k][g] = ld_relaxed(src + g);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NE; ++k) {
            if (!has[k]) continue;
            if (sign_bit(w[k])) {
                op_external<GC>(a, idx[k], w[k], (nz >> (16 + j[k])) & 1, G, acc);
                continue;
            }
#pragma unroll
            for (int g = 0; g < GM; ++g) {
                if (g < G) {
                    const uint32_t u = __float_as_uint(v[k][g]);
                    const float x = (u & 0x80000000u) == par ? __uint_as_float(u ^ par)
                                                             : op_wait(a, I + (size_t)idx[k] * G + g, fail);
                    acc[g] = fmaf(w[k], x, acc[g]);
                }
            }
        }
    }
#pragma unroll
    for (int off = LP / 2; off > 0; off >>= 1) {
#pragma unroll
        for (int g = 0; g < GM; ++g)
            if (g < G) acc[g] += __shfl_xor_sync(0xffffffffu, acc[g], off);
    }
    if (valid && !overflow && gl == 0 && !fail) {
        float* out = reinterpret_cast<float*>(a.I) + (size_t)dst * G;
        float val[GM];
#pragma unroll
        for (int g = 0; g < GM; ++g)
            if (g < G) val[g] = __uint_as_float(__float_as_uint(__fdividef(q[g].x + acc[g], P + q[g].y)) ^ par);
        if constexpr (GC == 4) {
            st_relaxed_v4(out, make_float4(val[0], val[1], val[2], val[3]));
        } else if constexpr (GC == 2) {
            st_relaxed_v2(out, make_float2(val[0], val[1]));
        } else {
#pragma unroll
            for (int g = 0; g < GM; ++g)
                if (g < G) st_relaxed(out + g, val[g]);
        }
    }
    return !fail;
}

template <int GC, int LP, typename ChunkFn>
__device__ __forceinline__ bool run_chunks_op(const SweepArgs& a, ChunkFn chunk, const float4* s_om, int grp, int gl,
                                              bool stall_here) {
    constexpr int CS = 32 / LP;  // tasks per warp step
    constexpr int PL = 8 / LP;
    constexpr int PF = 2;
    const uint64_t pol = policy_evict_first();
    auto pieces_of = [&](int64_t i) {
        OpPieces<LP> r;
        const int64_t k = chunk(i);
        const int4* src = a.op + (k * CS + grp) * 8 + gl * PL;
#pragma unroll
        for (int j = 0; j < PL; ++j) r.p[j] = k >= 0 ? ld_stream_int4(src + j, pol) : make_int4((int)TASK_PAD, 0, 0, 0);
        return r;
    };
    auto prefetch_chunk = [&](int64_t i) {
        const int64_t k = chunk(i);
        if (k >= 0 && (threadIdx.x & 31) == 0)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.op + k * CS * 8), "r"(CS * 128u));
    };
    OpPieces<LP> T[PF];
#pragma unroll
    for (int j = 0; j < PF; ++j) T[j] = pieces_of(j);
#pragma unroll
    for (int j = PF; j < 3 * PF; ++j) prefetch_chunk(j);
    for (int64_t i = 0; chunk(i) >= 0; ++i) {
        if ((i & 15) == 0 && __any_sync(0xffffffffu, ld_volatile_i32(a.err) != DEV_OK)) return false;
        const OpPieces<LP> t_new = pieces_of(i + PF);
        prefetch_chunk(i + 3 * PF);
        const bool stall = stall_here && i == 0 && grp == 0;
        bool overflow = false;
        bool good = op_task<GC, LP>(a, T[0], gl, stall, overflow);
        if (__any_sync(0xffffffffu, overflow)) {
            const int64_t k = chunk(i);
            const int4 tr = overflow ? __ldg(a.trec + k * CS + grp) : make_int4((int)TASK_PAD, 0, 0, 0);
            good = op_overflow<GC, LP>(a, tr, s_om, gl) && good;
        }
        if (__any_sync(0xffffffffu, !good)) return false;
#pragma unroll
        for (int j = 0; j < PF - 1; ++j) T[j] = T[j + 1];
        T[PF - 1] = t_new;
    }
    return true;
}

template <int GC, int LP>
__global__ void __launch_bounds__(256, SWEEP_REC_MINB) k_sweep_op(SweepArgs a) {
    extern __shared__ float4 s_om[];
    for (int i = threadIdx.x; i < a.nd; i += blockDim.x) s_om[i] = a.om32[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int grp = lane / LP, gl = lane % LP;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nchunks = a.n_chunks * LP;  // chunks of 32/LP tasks
    if (a.level_sync) {
        bool ok = true;
        for (int li = 0; li < a.n_levels; ++li) {
            const int64_t k0 = a.lev_chunk[li] * LP, k1 = a.lev_chunk[li + 1] * LP;
            if (ok) {
                auto chunk = [=](int64_t i) -> int64_t {
                    const int64_t k = k0 + warp + i * nwarps;
                    return k < k1 ? k : -1;
                };
                ok = run_chunks_op<GC, LP>(a, chunk, s_om, grp, gl, a.debug_stall && li == 0 && warp == 0);
            }
            if (!grid_sync(a.bar, gridDim.x, a.spin_budget, a.err)) return;
        }
    } else {
        auto chunk = [=](int64_t i) -> int64_t {
            const int64_t k = warp + i * nwarps;
            return k < nchunks ? k : -1;
        };
        run_chunks_op<GC, LP>(a, chunk, s_om, grp, gl, a.debug_stall && warp == 0);
    }
}

// Lean form for one frequency group and 8 lanes per task (dataflow schedule). A warp takes 4 tasks
// (512 contiguous bytes of operator lines) per step, the lines of the next two steps in flight in
// registers and those of the three after in L2 (bulk prefetch). Lane 0 of a task holds its header,
// lanes 1..7 two entries each. The common case -- an interior upwind value already written by this
// sweep -- is a load, a sign test and an FMA; periodic and boundary inflow stay inline; only a wait
// for a value not yet written goes out of line. A failed wait sets the device error word, which the
// loop checks every 16 steps.
__global__ void __launch_bounds__(256, SWEEP_REC_MINB) k_sweep_op1(SweepArgs a) {
    extern __shared__ float4 s_om[];
    for (int i = threadIdx.x; i < a.nd; i += blockDim.x) s_om[i] = a.om32[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int grp = lane >> 3, gl = lane & 7, lead = lane & ~7;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nchunks = a.n_chunks * 8;  // steps of 4 tasks
    const uint64_t pol = policy_evict_first();
    const float* I = reinterpret_cast<const float*>(a.I);
    const float2* cm = reinterpret_cast<const float2*>(a.cm);
    const uint32_t par = a.parity ? 0x80000000u : 0u;
    const int4 pad = make_int4((int)TASK_PAD, 0, 0, 0);
    const int4* src = a.op + warp * 32 + lane;  // this lane's 16 bytes of step k: src + (k - warp) * 32
    const int64_t stride = nwarps * 32;
    int64_t k = warp;
    int4 cur = k < nchunks ? ld_stream_int4(src, pol) : pad;
    int4 nxt = k + nwarps < nchunks ? ld_stream_int4(src + stride, pol) : pad;
    if (lane == 0)
        for (int j = 2; j <= 4; ++j)
            if (k + j * nwarps < nchunks)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.op + (k + j * nwarps) * 32),
                             "r"(512u));
    if (a.debug_stall && warp == 0 && lane == 0) {  // test hook: a wait on a word that nothing writes
        float dummy;
        wait_value(reinterpret_cast<const float*>(a.stall_word), 1, a, dummy);
    }
    for (int64_t i = 0; k < nchunks; ++i, k += nwarps) {
        if ((i & 15) == 0 && __any_sync(0xffffffffu, ld_volatile_i32(a.err) != DEV_OK)) return;
        src += stride;
        const int4 nn = k + 2 * nwarps < nchunks ? ld_stream_int4(src + stride, pol) : pad;
        if (lane == 0 && k + 5 * nwarps < nchunks)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.op + (k + 5 * nwarps) * 32), "r"(512u));
        const uint32_t e = (uint32_t)__shfl_sync(0xffffffffu, cur.x, lead);
        const int nz = __shfl_sync(0xffffffffu, cur.z, lead);
        const int nin = nz & 0xff;
        const bool valid = e != TASK_PAD;
        const bool over = valid && nin > OP_MAX;
        const bool work = valid && !over;
        bool fail = false;
        float acc = 0.f;
        float2 q = make_float2(0.f, 1.f);
        if (gl == 0) {
            if (work) q = cm[e & a.cmask];
        } else if (work) {
            const int j0 = 2 * gl - 2;
            const bool h0 = j0 < nin, h1 = j0 + 1 < nin;
            const bool in0 = h0 && cur.y >= 0, in1 = h1 && cur.w >= 0;  // sign bit clear: interior entry
            const float x0 = in0 ? ld_relaxed(I + (uint32_t)cur.x) : 0.f;
            const float x1 = in1 ? ld_relaxed(I + (uint32_t)cur.z) : 0.f;
            const float w0 = __int_as_float(cur.y), w1 = __int_as_float(cur.w);
            if (in0) {
                const uint32_t u = __float_as_uint(x0);
                acc = w0 * ((u & 0x80000000u) == par ? __uint_as_float(u ^ par) : op_wait(a, I + (uint32_t)cur.x, fail));
            } else if (h0) {
                op_external<1>(a, (uint32_t)cur.x, w0, (nz >> (16 + j0)) & 1, 1, &acc);
            }
            if (in1) {
                const uint32_t u = __float_as_uint(x1);
                acc = fmaf(w1, (u & 0x80000000u) == par ? __uint_as_float(u ^ par) : op_wait(a, I + (uint32_t)cur.z, fail),
                           acc);
            } else if (h1) {
                op_external<1>(a, (uint32_t)cur.z, w1, (nz >> (17 + j0)) & 1, 1, &acc);
            }
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (gl == 0 && work && !fail) {
            const float val = __fdividef(q.x + acc, __int_as_float(cur.y) + q.y);
            st_relaxed(reinterpret_cast<float*>(a.I) + (uint32_t)cur.w, __uint_as_float(__float_as_uint(val) ^ par));
        }
        if (__any_sync(0xffffffffu, over)) {
            const int4 tr = over ? __ldg(a.trec + k * 4 + grp) : pad;
            op_overflow<1, 8>(a, tr, s_om, gl);  // a failed wait inside sets the error word
        }
        cur = nxt;
        nxt = nn;
    }
}

// Two tasks per lane group per step: a warp takes 8 tasks (1 KB of operator lines) per loop
// iteration, lanes gl of group grp holding piece gl of tasks 8k+grp and 8k+4+grp. The fixed cost
// of an iteration (line loads, prefetch, header shuffles, loop control, the overflow vote) is shared
// by twice as many tasks as in k_sweep_op1, and each lane has up to four upwind reads in flight.
// The 8 tasks of a step lie in one level (levels are padded to 32 tasks), so they are independent.
// Operator lines stream through L2 marked evict-first, intensities are read and written evict-last.
__global__ void __launch_bounds__(256, SWEEP_REC_MINB) k_sweep_op2(SweepArgs a) {
    extern __shared__ float4 s_om[];
    for (int i = threadIdx.x; i < a.nd; i += blockDim.x) s_om[i] = a.om32[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int grp = lane >> 3, gl = lane & 7, lead = lane & ~7;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nsteps = a.n_chunks * 4;  // steps of 8 tasks
    const uint64_t pol = policy_evict_first();
    const uint64_t keep = policy_evict_last();  // intensities: each is read again by ~8 downwind tasks
    const float* I = reinterpret_cast<const float*>(a.I);
    const float2* cm = reinterpret_cast<const float2*>(a.cm);
    const uint32_t par = a.parity ? 0x80000000u : 0u;
    const int4 pad = make_int4((int)TASK_PAD, 0, 0, 0);
    const int4* src = a.op + warp * 64 + lane;  // step k: tasks A at src + (k-warp)*64, B 32 int4 further
    const int64_t stride = nwarps * 64;
    int64_t k = warp;
    int4 ca = k < nsteps ? ld_stream_int4(src, pol) : pad;
    int4 cb = k < nsteps ? ld_stream_int4(src + 32, pol) : pad;
    if (lane == 0)
        for (int j = 1; j <= 2; ++j)
            if (k + j * nwarps < nsteps)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.op + (k + j * nwarps) * 64),
                             "r"(1024u));
    if (a.debug_stall && warp == 0 && lane == 0) {  // test hook: a wait on a word that nothing writes
        float dummy;
        wait_value(reinterpret_cast<const float*>(a.stall_word), 1, a, dummy);
    }
    for (int64_t i = 0; k < nsteps; ++i, k += nwarps) {
        if ((i & 15) == 0 && __any_sync(0xffffffffu, ld_volatile_i32(a.err) != DEV_OK)) return;
        src += stride;
        const bool more = k + nwarps < nsteps;
        const int4 na = more ? ld_stream_int4(src, pol) : pad;
        const int4 nb = more ? ld_stream_int4(src + 32, pol) : pad;
        if (lane == 0 && k + 3 * nwarps < nsteps)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.op + (k + 3 * nwarps) * 64), "r"(1024u));
        const uint32_t ea = (uint32_t)__shfl_sync(0xffffffffu, ca.x, lead);
        const uint32_t eb = (uint32_t)__shfl_sync(0xffffffffu, cb.x, lead);
        const int za = __shfl_sync(0xffffffffu, ca.z, lead);
        const int zb = __shfl_sync(0xffffffffu, cb.z, lead);
        const int nina = za & 0xff, ninb = zb & 0xff;
        const bool overa = ea != TASK_PAD && nina > OP_MAX, overb = eb != TASK_PAD && ninb > OP_MAX;
        const bool worka = ea != TASK_PAD && !overa, workb = eb != TASK_PAD && !overb;
        bool fail = false;
        float acca = 0.f, accb = 0.f;
        float2 qa = make_float2(0.f, 1.f), qb = make_float2(0.f, 1.f);
        if (gl == 0) {
            if (worka) qa = cm[ea & a.cmask];
            if (workb) qb = cm[eb & a.cmask];
        } else {
            const int j0 = 2 * gl - 2;
            const bool ha0 = worka && j0 < nina, ha1 = worka && j0 + 1 < nina;
            const bool hb0 = workb && j0 < ninb, hb1 = workb && j0 + 1 < ninb;
            const bool ia0 = ha0 && ca.y >= 0, ia1 = ha1 && ca.w >= 0;  // sign bit clear: interior entry
            const bool ib0 = hb0 && cb.y >= 0, ib1 = hb1 && cb.w >= 0;
            const float xa0 = ia0 ? ld_relaxed_hint(I + (uint32_t)ca.x, keep) : 0.f;
            const float xa1 = ia1 ? ld_relaxed_hint(I + (uint32_t)ca.z, keep) : 0.f;
            const float xb0 = ib0 ? ld_relaxed_hint(I + (uint32_t)cb.x, keep) : 0.f;
            const float xb1 = ib1 ? ld_relaxed_hint(I + (uint32_t)cb.z, keep) : 0.f;
            auto term = [&](bool in, bool has, float x, uint32_t idx, int wbits, int bit, int z) -> float {
                const float w = __int_as_float(wbits);
                if (in) {
                    const uint32_t u = __float_as_uint(x);
                    return w * ((u & 0x80000000u) == par ? __uint_as_float(u ^ par) : op_wait(a, I + idx, fail));
                }
                float t = 0.f;
                if (has) op_external<1>(a, idx, w, (z >> (16 + bit)) & 1, 1, &t);
                return t;
            };
            acca = term(ia0, ha0, xa0, (uint32_t)ca.x, ca.y, j0, za) + term(ia1, ha1, xa1, (uint32_t)ca.z, ca.w, j0 + 1, za);
            accb = term(ib0, hb0, xb0, (uint32_t)cb.x, cb.y, j0, zb) + term(ib1, hb1, xb1, (uint32_t)cb.z, cb.w, j0 + 1, zb);
        }
        acca += __shfl_xor_sync(0xffffffffu, acca, 4);
        accb += __shfl_xor_sync(0xffffffffu, accb, 4);
        acca += __shfl_xor_sync(0xffffffffu, acca, 2);
        accb += __shfl_xor_sync(0xffffffffu, accb, 2);
        acca += __shfl_xor_sync(0xffffffffu, acca, 1);
        accb += __shfl_xor_sync(0xffffffffu, accb, 1);
        if (gl == 0 && !fail) {
            float* out = reinterpret_cast<float*>(a.I);
            if (worka) {
                const float v = __fdividef(qa.x + acca, __int_as_float(ca.y) + qa.y);
                st_relaxed_hint(out + (uint32_t)ca.w, __uint_as_float(__float_as_uint(v) ^ par), keep);
            }
            if (workb) {
                const float v = __fdividef(qb.x + accb, __int_as_float(cb.y) + qb.y);
                st_relaxed_hint(out + (uint32_t)cb.w, __uint_as_float(__float_as_uint(v) ^ par), keep);
            }
        }
        if (__any_sync(0xffffffffu, overa || overb)) {  // a failed wait inside sets the error word
            if (__any_sync(0xffffffffu, overa)) op_overflow<1, 8>(a, overa ? __ldg(a.trec + k * 8 + grp) : pad, s_om, gl);
            if (__any_sync(0xffffffffu, overb)) op_overflow<1, 8>(a, overb ? __ldg(a.trec + k * 8 + 4 + grp) : pad, s_om, gl);
        }
        ca = na;
        cb = nb;
    }
}

// ---------------------------------------------------------------------------------------------
// FP32 forward sweep over the packed operator (see pack_plan / k_pack): one warp per packet of 32
// lanes x two entry slots, PK packets per warp step. Every lane decodes its own slots and gathers its
// upwind values (interior: this sweep's intensities, with the readiness test on the sign bit;
// periodic: the previous iteration's; boundary: the inflow array) with no branch on the entry kind;
// a segmented shuffle scan (segments = tasks; 4 steps, a 5th in packets holding a task of more than 16
// lanes) sums each task's inflow into its head lane, which solves the cell balance
// (P_c + kappa_t V) I = q + sum |a| I_up and stores it. Only a wait for a value not yet written leaves
// the straight line.
// ---------------------------------------------------------------------------------------------
template <int GC>
__device__ __forceinline__ void pk_gather(const float* p, bool has, uint64_t pol, float* x) {
    if constexpr (GC == 4) {
        const float4 v = ld_relaxed_hint_v4_if(p, pol, has);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else if constexpr (GC == 2) {
        const float2 v = ld_relaxed_hint_v2_if(p, pol, has);
        x[0] = v.x; x[1] = v.y;
    } else {
        x[0] = ld_relaxed_hint_if(p, pol, has);
    }
}

// one packet's decoded state between the gather and the solve
template <int GC>
struct PkLane {
    int4 s;           // this lane's two slots
    bool h0, h1;      // slot holds an entry whose source exists
    bool in0, in1;    // interior entry (readiness tested)
    bool head;
    bool lng;         // the packet holds a task of more than 16 lanes
    int pos;          // rank of this lane within its task
    float x0[GC], x1[GC];
    float q[2 * GC];  // head lane: {q, kappa_t V} per group
};

// source of a slot: this sweep's intensities, the previous iteration's (periodic) or the boundary inflow
__device__ __forceinline__ const float* pk_base(const SweepArgs& a, int idx, int w) {
    return w >= 0 ? reinterpret_cast<const float*>(a.I)
                  : ((uint32_t)idx & PK_BOUNDARY ? reinterpret_cast<const float*>(a.bc)
                                                 : reinterpret_cast<const float*>(a.Iprev));
}

template <int GC>
__device__ __forceinline__ void pk_decode(const SweepArgs& a, const int4 s, const uint2 m, int lane, uint64_t keep,
                                          PkLane<GC>& t) {
    t.s = s;
    t.head = (m.x >> lane) & 1u;
    t.lng = m.y != 0u;
    const unsigned hb = m.x & ((1u << lane) - 1u);
    t.pos = lane - (hb ? 32 - __clz(hb) : 0);
    t.in0 = s.y >= 0;
    t.in1 = s.w >= 0 && !t.head;
    const float* b0 = pk_base(a, s.x, s.y);
    const float* b1 = pk_base(a, s.z, s.w);
    t.h0 = ((uint32_t)s.y << 1) != 0u && b0 != nullptr;
    t.h1 = !t.head && ((uint32_t)s.w << 1) != 0u && b1 != nullptr;
    pk_gather<GC>(b0 + (size_t)((uint32_t)s.x & ~PK_BOUNDARY) * GC, t.h0, keep, t.x0);
    pk_gather<GC>(b1 + (size_t)((uint32_t)s.z & ~PK_BOUNDARY) * GC, t.h1, keep, t.x1);
    // the cell's source and kappa_t V (head lanes), loaded beside the gathers
    const float2* cm = reinterpret_cast<const float2*>(a.cm) + (size_t)((uint32_t)s.z & a.cmask) * GC;
    if constexpr (GC == 1) {
        const float2 v = ld_nc_v2_if(cm, t.head);
        t.q[0] = v.x; t.q[1] = v.y;
    } else {
#pragma unroll
        for (int h = 0; h < GC / 2; ++h) {
            const float4 v = ld_nc_v4_if(cm + 2 * h, t.head);
            t.q[4 * h] = v.x; t.q[4 * h + 1] = v.y; t.q[4 * h + 2] = v.z; t.q[4 * h + 3] = v.w;
        }
    }
}

// any of a slot's GC values lacks this sweep's parity
template <int GC>
__device__ __forceinline__ bool pk_slot_unready(const float* x, uint32_t par) {
    uint32_t m = 0u;
#pragma unroll
    for (int g = 0; g < GC; ++g) m |= __float_as_uint(x[g]) ^ par;
    return m >> 31;
}

// sign bit of any gathered interior value differs from this sweep's parity: not written yet
template <int GC>
__device__ __forceinline__ bool pk_unready(const PkLane<GC>& t, uint32_t par) {
    return (t.h0 && t.in0 && pk_slot_unready<GC>(t.x0, par)) | (t.h1 && t.in1 && pk_slot_unready<GC>(t.x1, par));
}

// re-read of a slot's GC values (one vector load) where `on`, keeping them otherwise
template <int GC>
__device__ __forceinline__ void pk_reload(const float* p, bool on, float* x) {
    if constexpr (GC == 4) ld_relaxed_keep_v4_if(p, on, x);
    else if constexpr (GC == 2) ld_relaxed_keep_v2_if(p, on, x);
    else x[0] = ld_relaxed_keep_if(p, on, x[0]);
}

// The step's gathered interior values not yet written by this sweep: all of them are re-read together,
// one round trip per poll (a slot's GC values as one vector load), until every one carries this
// sweep's parity (a serial wait per value would cost a round trip per value after its producer
// finished). Bounded: after spin_budget polls, or when another warp has set the device error word, the
// step gives up and the error word is set.
template <int GC, int PK>
__device__ __forceinline__ void pk_wait_all(const SweepArgs& a, PkLane<GC> (&t)[PK], uint32_t par, bool& fail) {
    const float* I = reinterpret_cast<const float*>(a.I);
    for (long long n = 0;; ++n) {
        bool nr = false;
#pragma unroll
        for (int p = 0; p < PK; ++p) {
            const bool u0 = t[p].h0 && t[p].in0 && pk_slot_unready<GC>(t[p].x0, par);
            const bool u1 = t[p].h1 && t[p].in1 && pk_slot_unready<GC>(t[p].x1, par);
            pk_reload<GC>(I + (size_t)(uint32_t)t[p].s.x * GC, u0, t[p].x0);
            pk_reload<GC>(I + (size_t)(uint32_t)t[p].s.z * GC, u1, t[p].x1);
        }
#pragma unroll
        for (int p = 0; p < PK; ++p) nr |= pk_unready<GC>(t[p], par);
        if (!__any_sync(0xffffffffu, nr)) return;
        if (n >= a.spin_budget || ((n & 63) == 63 && ld_volatile_i32(a.err) != DEV_OK)) {
            atomicCAS(a.err, DEV_OK, DEV_TIMEOUT);
            fail = true;
            return;
        }
        __nanosleep(20);
    }
}

// segmented sum over each task's lanes, then the head lane solves and stores the cell: the balance
// (q + sum) / (P_c + kappa_t V), the EXP law (intensity and cell mean), or the transposed balance
// (w_d q + sum) / (P_c + kappa_t V) of the adjoint sweep
template <int GC, int MODE>
__device__ __forceinline__ void pk_solve(const SweepArgs& a, const PkLane<GC>& t, uint32_t par, uint64_t keep,
                                         bool fail) {
    const float w0 = fabsf(__int_as_float(t.s.y)), w1 = fabsf(__int_as_float(t.s.w));
    float acc[GC];
#pragma unroll
    for (int g = 0; g < GC; ++g) acc[g] = fmaf(w1, fabsf(t.x1[g]), w0 * fabsf(t.x0[g]));
#pragma unroll
    for (int off = 1; off < 16; off <<= 1) {
#pragma unroll
        for (int g = 0; g < GC; ++g) {
            const float y = __shfl_up_sync(0xffffffffu, acc[g], off);
            if (t.pos >= off) acc[g] += y;
        }
    }
    if (t.lng) {  // warp-uniform: a task spans more than 16 lanes
#pragma unroll
        for (int g = 0; g < GC; ++g) {
            const float y = __shfl_up_sync(0xffffffffu, acc[g], 16);
            if (t.pos >= 16) acc[g] += y;
        }
    }
    // head lanes solve and store their cell (predicated: no branch, the other lanes skip the store)
    const bool on = t.head && !fail;
    const uint32_t e = (uint32_t)t.s.z;
    const uint32_t dst = (e >> a.cshift) * (uint32_t)a.N + (e & a.cmask);
    const float P = __int_as_float(t.s.w);
    float v[GC];
    if constexpr (MODE == PK_EXP) {
        float m[GC];
#pragma unroll
        for (int g = 0; g < GC; ++g) {
            exp_update_lanes(acc[g], t.q[2 * g], t.q[2 * g + 1], P, v[g], m[g]);
            v[g] = __uint_as_float(__float_as_uint(v[g]) ^ par);
        }
        float* mo = reinterpret_cast<float*>(a.Imean) + (size_t)dst * GC;
        if constexpr (GC == 4) st_relaxed_hint_v4_if(mo, make_float4(m[0], m[1], m[2], m[3]), keep, on);
        else if constexpr (GC == 2) st_relaxed_hint_v2_if(mo, make_float2(m[0], m[1]), keep, on);
        else st_relaxed_hint_if(mo, m[0], keep, on);
    } else {
        float wd = 1.f;
        if constexpr (MODE == PK_TRANSPOSED) wd = (float)__ldg(a.w64 + (t.head ? (e >> a.cshift) : 0u));
#pragma unroll
        for (int g = 0; g < GC; ++g) {
            const float src = MODE == PK_TRANSPOSED ? wd * t.q[2 * g] : t.q[2 * g];
            v[g] = __uint_as_float(__float_as_uint(__fdividef(src + acc[g], P + t.q[2 * g + 1])) ^ par);
        }
    }
    float* out = reinterpret_cast<float*>(a.I) + (size_t)dst * GC;
    if constexpr (GC == 4) st_relaxed_hint_v4_if(out, make_float4(v[0], v[1], v[2], v[3]), keep, on);
    else if constexpr (GC == 2) st_relaxed_hint_v2_if(out, make_float2(v[0], v[1]), keep, on);
    else st_relaxed_hint_if(out, v[0], keep, on);
}

// Steps [k0, k1) of PK packets, warp w taking k0 + w, k0 + w + W, ...; the packets of the next step
// are loaded one step ahead into registers and those three steps ahead prefetched into L2.
template <int GC, int PK, int MODE>
__device__ __forceinline__ bool pk_steps(const SweepArgs& a, int64_t k0, int64_t k1, int64_t warp, int64_t nwarps) {
    const int lane = threadIdx.x & 31;
    const uint64_t pol = policy_evict_first();
    const uint64_t keep = policy_evict_last();  // intensities: each is read again by ~8 downwind tasks
    const uint32_t par = a.parity ? 0x80000000u : 0u;
    const int4 zero = make_int4(0, 0, 0, 0);
    int64_t k = k0 + warp;
    int4 cur[PK];
    uint2 cm_[PK];
    auto load = [&](int64_t kk, int4* s, uint2* m) {
        const bool ok = kk < k1;
#pragma unroll
        for (int p = 0; p < PK; ++p) {
            s[p] = ok ? ld_stream_int4(a.pk + (kk * PK + p) * 32 + lane, pol) : zero;
            m[p] = ok ? __ldg(a.pk_meta + kk * PK + p) : make_uint2(0u, 0u);
        }
    };
    load(k, cur, cm_);
    if (lane == 0)
        for (int j = 1; j <= 2; ++j)
            if (k + j * nwarps < k1)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.pk + (k + j * nwarps) * PK * 32),
                             "r"(PK * 512u));
    for (int64_t i = 0; k < k1; ++i, k += nwarps) {
        if ((i & 15) == 0 && __any_sync(0xffffffffu, ld_volatile_i32(a.err) != DEV_OK)) return false;
        int4 nxt[PK];
        uint2 nm[PK];
        load(k + nwarps, nxt, nm);
        if (lane == 0 && k + 3 * nwarps < k1)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.pk + (k + 3 * nwarps) * PK * 32),
                         "r"(PK * 512u));
        PkLane<GC> t[PK];
#pragma unroll
        for (int p = 0; p < PK; ++p) pk_decode<GC>(a, cur[p], cm_[p], lane, keep, t[p]);
        bool fail = false;
        bool nr = false;
#pragma unroll
        for (int p = 0; p < PK; ++p) nr |= pk_unready<GC>(t[p], par);
        if (__any_sync(0xffffffffu, nr)) pk_wait_all<GC, PK>(a, t, par, fail);
#pragma unroll
        for (int p = 0; p < PK; ++p) pk_solve<GC, MODE>(a, t[p], par, keep, fail);
#pragma unroll
        for (int p = 0; p < PK; ++p) {
            cur[p] = nxt[p];
            cm_[p] = nm[p];
        }
    }
    return true;
}

// resident 256-thread blocks per SM the packed kernel is compiled for (64 registers; 3 with two packets
// per step and four groups, or two groups under the EXP law, whose state needs more)
template <int GC, int PK, int MODE>
struct PkMinBlocks {
    static constexpr int value = (PK == 2 && (GC == 4 || (GC == 2 && MODE == PK_EXP))) ? 3 : 4;
};

template <int GC, int PK, int MODE>
__global__ void __launch_bounds__(256, (PkMinBlocks<GC, PK, MODE>::value)) k_sweep_pk(const __grid_constant__ SweepArgs a) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (a.debug_stall && warp == 0 && (threadIdx.x & 31) == 0) {  // test hook: a wait on a word nothing writes
        float dummy;
        wait_value(reinterpret_cast<const float*>(a.stall_word), 1, a, dummy);
    }
    if (a.level_sync) {
        for (int li = 0; li < a.n_levels; ++li) {
            pk_steps<GC, PK, MODE>(a, a.lev_pk[li] / PK, a.lev_pk[li + 1] / PK, warp, nwarps);
            if (!grid_sync(a.bar, gridDim.x, a.spin_budget, a.err)) return;
        }
    } else {
        pk_steps<GC, PK, MODE>(a, 0, a.n_pk / PK, warp, nwarps);
    }
}

// the packed kernel of a launch: groups (1, 2 or 4; the transposed sweep's 2G split groups: 2 or 4),
// packets per warp step and cell update
template <int PK>
const void* pk_kernel(int G, int mode) {
    if (mode == PK_TRANSPOSED) return G == 2 ? (const void*)k_sweep_pk<2, PK, PK_TRANSPOSED>
                                             : (const void*)k_sweep_pk<4, PK, PK_TRANSPOSED>;
    if (mode == PK_EXP) {
        switch (G) {
            case 1: return (const void*)k_sweep_pk<1, PK, PK_EXP>;
            case 2: return (const void*)k_sweep_pk<2, PK, PK_EXP>;
            default: return (const void*)k_sweep_pk<4, PK, PK_EXP>;
        }
    }
    switch (G) {
        case 1: return (const void*)k_sweep_pk<1, PK, PK_BALANCE>;
        case 2: return (const void*)k_sweep_pk<2, PK, PK_BALANCE>;
        default: return (const void*)k_sweep_pk<4, PK, PK_BALANCE>;
    }
}

template <int PK>
cudaError_t launch_pk(const SweepArgs& a, const cudaLaunchConfig_t& cfg, int mode) {
    void* args[] = {(void*)&a};
    return cudaLaunchKernelExC(&cfg, pk_kernel<PK>(a.G, mode), args);
}

template <int PK>
int occupancy_pk(int G, int mode, int threads, size_t smem) {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pk_kernel<PK>(G, mode), threads, smem);
    return n;
}

template <int LP>
cudaError_t launch_op_lanes(const SweepArgs& a, const cudaLaunchConfig_t& cfg) {
    if (LP == 8 && a.G == 1 && !a.level_sync) return cudaLaunchKernelEx(&cfg, k_sweep_op1, a);
    switch (a.G) {
        case 1: return cudaLaunchKernelEx(&cfg, k_sweep_op<1, LP>, a);
        case 2: return cudaLaunchKernelEx(&cfg, k_sweep_op<2, LP>, a);
        case 4: return cudaLaunchKernelEx(&cfg, k_sweep_op<4, LP>, a);
        default: return cudaLaunchKernelEx(&cfg, k_sweep_op<0, LP>, a);
    }
}

template <int LP>
int occupancy_op(int G, int threads, size_t smem) {
    int n = 0;
    if (LP == 8 && G == 1) {  // the lean kernel (dataflow) has the same launch bounds as the general one
        int n1 = 0, n2 = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n1, k_sweep_op1, threads, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n2, k_sweep_op<1, 8>, threads, smem);
        return n1 < n2 ? n1 : n2;
    }
    switch (G) {
        case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_op<1, LP>, threads, smem); break;
        case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_op<2, LP>, threads, smem); break;
        case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_op<4, LP>, threads, smem); break;
        default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_op<0, LP>, threads, smem); break;
    }
    return n;
}

// ---------------------------------------------------------------------------------------------
// K8: the plain path -- one launch per (direction, level) segment, FP64, one thread per task
// walking its face sides in order (the oracle's summation order).
// ---------------------------------------------------------------------------------------------
template <int GC>
__device__ __forceinline__ void plain_task(const SweepArgs& a, uint32_t entry) {
    constexpr int GM = GC > 0 ? GC : 8;
    const int G = GC > 0 ? GC : a.G;
    const uint32_t c = entry & a.cmask;
    const uint32_t dl = entry >> a.cshift;
    const uint32_t r0 = a.rowptr[c], r1 = a.rowptr[c + 1];
    const double* om64 = a.om64 + 3 * dl;
    const double2* cm = reinterpret_cast<const double2*>(a.cm) + (size_t)c * G;
    double* I = reinterpret_cast<double*>(a.I);
    const size_t slab = (size_t)dl * a.N;
    double acc[GM];
    for (int g = 0; g < GM; ++g)  // EXP keeps the inflow apart from the source
        if (g < G) acc[g] = a.law ? 0.0 : (a.reverse ? __dmul_rn(a.w64[dl], cm[g].x) : cm[g].x);
    double P = 0.0;
    for (uint32_t s = r0; s < r1; ++s) {
        const int32_t nb = a.side[s].x;
        const d4 n = a.side64[s];
        const double t = exact_t(n, om64);
        if (t == 0.0) continue;
        const double w = __dmul_rn(n.w, fabs(t));
        if (t > 0.0) P = __dadd_rn(P, w);
        const bool inflow = a.reverse ? t > 0.0 : t < 0.0;
        if (!inflow) continue;
        double wi = w;
        if (a.dc_mask && nb >= 0) {  // scheme (b): the upwind cell's share, if it chose this face
            const int64_t i = (int64_t)(nb & NBR_MASK) * a.nd + dl;
            if (!((a.dc_mask[i] >> a.twin[s]) & 1ull)) continue;
            wi = a.dc_share64[i];
        }
        const double* src = nullptr;
        if (nb >= 0 && !(nb & NBR_PERIODIC)) src = I + (slab + (uint32_t)nb) * G;
        else if (nb >= 0) src = a.Iprev ? reinterpret_cast<const double*>(a.Iprev) + (slab + (nb & NBR_MASK)) * G
                                        : nullptr;
        else if (a.reverse) continue;
        else src = a.bc ? reinterpret_cast<const double*>(a.bc) + (size_t)(-1 - nb) * G : nullptr;
        if (!src) continue;
        for (int g = 0; g < GM; ++g)
            if (g < G) acc[g] = __dadd_rn(acc[g], __dmul_rn(wi, fabs(src[g])));
    }
    double* dst = I + (slab + c) * G;
    for (int g = 0; g < GM; ++g) {
        if (g < G) {
            double v;
            if (a.law) {
                double mean;
                exp_law(acc[g], cm[g].x, cm[g].y, P, v, mean);
                reinterpret_cast<double*>(a.Imean)[(slab + c) * G + g] = mean;
            } else {
                v = __ddiv_rn(acc[g], __dadd_rn(P, cm[g].y));
            }
            dst[g] = a.parity ? -v : v;
        }
    }
}

template <int GC>
__global__ void __launch_bounds__(256) k_plain(SweepArgs a, uint32_t begin, uint32_t end) {
    const uint32_t i = begin + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= end) return;
    plain_task<GC>(a, a.task[i]);
}

template <typename real, int L>
cudaError_t launch_lanes(const SweepArgs& a, const cudaLaunchConfig_t& cfg) {
    switch (a.G) {
        case 1: return cudaLaunchKernelEx(&cfg, k_sweep<real, 1, L>, a);
        case 2: return cudaLaunchKernelEx(&cfg, k_sweep<real, 2, L>, a);
        case 4: return cudaLaunchKernelEx(&cfg, k_sweep<real, 4, L>, a);
        default: return cudaLaunchKernelEx(&cfg, k_sweep<real, 0, L>, a);
    }
}

template <int L>
cudaError_t launch_rec_lanes(const SweepArgs& a, const cudaLaunchConfig_t& cfg) {
    switch (a.G) {
        case 1: return cudaLaunchKernelEx(&cfg, k_sweep_rec<1, L>, a);
        case 2: return cudaLaunchKernelEx(&cfg, k_sweep_rec<2, L>, a);
        case 4: return cudaLaunchKernelEx(&cfg, k_sweep_rec<4, L>, a);
        default: return cudaLaunchKernelEx(&cfg, k_sweep_rec<0, L>, a);
    }
}

template <int L>
int occupancy_rec_lanes(int G, int threads, size_t smem) {
    int n = 0;
    switch (G) {
        case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_rec<1, L>, threads, smem); break;
        case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_rec<2, L>, threads, smem); break;
        case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_rec<4, L>, threads, smem); break;
        default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_rec<0, L>, threads, smem); break;
    }
    return n;
}

template <typename real>
cudaError_t launch_typed(const SweepArgs& a, int blocks, int threads, cudaStream_t st, int* kid) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = sizeof(float4) * (size_t)a.nd;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (sizeof(real) == 4 && a.pk) {  // FP32 over the packed operator (forward or transposed)
        *kid = SWEEP_KERNEL_PACKED;
        const int mode = a.reverse ? PK_TRANSPOSED : (a.law ? PK_EXP : PK_BALANCE);
        return a.lanes >= 64 ? launch_pk<2>(a, cfg, mode) : launch_pk<1>(a, cfg, mode);
    }
    if (sizeof(real) == 4 && !a.reverse && a.op) {  // FP32 forward over the assembled operator
        if (a.lanes == 16 && a.G == 1 && !a.level_sync) {
            *kid = SWEEP_KERNEL_OPERATOR_PAIR;
            return cudaLaunchKernelEx(&cfg, k_sweep_op2, a);
        }
        *kid = a.lanes >= 8 && a.G == 1 && !a.level_sync ? SWEEP_KERNEL_OPERATOR_LEAN : SWEEP_KERNEL_OPERATOR;
        if (a.lanes <= 2) return launch_op_lanes<2>(a, cfg);
        if (a.lanes == 4) return launch_op_lanes<4>(a, cfg);
        return launch_op_lanes<8>(a, cfg);
    }
    if (sizeof(real) == 4 && !a.reverse && !a.law && !a.dc_mask) {  // FP32 forward, scheme (a): the record kernel
        *kid = SWEEP_KERNEL_RECORDS;
        if (a.lanes == 1) return launch_rec_lanes<1>(a, cfg);
        if (a.lanes == 2) return launch_rec_lanes<2>(a, cfg);
        if (a.lanes == 4) return launch_rec_lanes<4>(a, cfg);
        return launch_rec_lanes<8>(a, cfg);
    }
    *kid = SWEEP_KERNEL_GEOMETRY;
    if (a.lanes == 16) return launch_lanes<real, 16>(a, cfg);
    if (a.lanes == 2) return launch_lanes<real, 2>(a, cfg);
    if (a.lanes == 1) return launch_lanes<real, 1>(a, cfg);
    if (a.lanes == 8) return launch_lanes<real, 8>(a, cfg);
    return launch_lanes<real, 4>(a, cfg);
}

template <typename real, int L>
int occupancy_lanes(int G, int threads, size_t smem) {
    int n = 0;
    switch (G) {
        case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<real, 1, L>, threads, smem); break;
        case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<real, 2, L>, threads, smem); break;
        case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<real, 4, L>, threads, smem); break;
        default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<real, 0, L>, threads, smem); break;
    }
    return n;
}

}  // namespace

int sweep_occupancy(int precision, int G, int threads, int nd, int lanes, int generic, int fmt, int pk_mode) {
    size_t smem = sizeof(float4) * (size_t)nd;
    if (precision == 32 && fmt == OPF_PACKETS)
        return lanes >= 64 ? occupancy_pk<2>(G, pk_mode, threads, smem) : occupancy_pk<1>(G, pk_mode, threads, smem);
    const int reverse = generic;
    if (precision == 32 && !reverse && fmt == OPF_LINES) {
        if (lanes == 16 && G == 1) {
            int n = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_op2, threads, smem);
            return n;
        }
        if (lanes <= 2) return occupancy_op<2>(G, threads, smem);
        if (lanes == 4) return occupancy_op<4>(G, threads, smem);
        return occupancy_op<8>(G, threads, smem);
    }
    if (precision == 32 && !reverse) {
        if (lanes == 1) return occupancy_rec_lanes<1>(G, threads, smem);
        if (lanes == 2) return occupancy_rec_lanes<2>(G, threads, smem);
        if (lanes == 4) return occupancy_rec_lanes<4>(G, threads, smem);
        return occupancy_rec_lanes<8>(G, threads, smem);
    }
    if (precision == 64) {
        if (lanes == 16) return occupancy_lanes<double, 16>(G, threads, smem);
        if (lanes == 2) return occupancy_lanes<double, 2>(G, threads, smem);
        if (lanes == 1) return occupancy_lanes<double, 1>(G, threads, smem);
        return lanes == 8 ? occupancy_lanes<double, 8>(G, threads, smem) : occupancy_lanes<double, 4>(G, threads, smem);
    }
    if (lanes == 16) return occupancy_lanes<float, 16>(G, threads, smem);
    if (lanes == 2) return occupancy_lanes<float, 2>(G, threads, smem);
    if (lanes == 1) return occupancy_lanes<float, 1>(G, threads, smem);
    return lanes == 8 ? occupancy_lanes<float, 8>(G, threads, smem) : occupancy_lanes<float, 4>(G, threads, smem);
}

cudaError_t launch_sweep(const SweepArgs& a, int precision, int blocks, int threads, cudaStream_t st, int* kernel) {
    int kid = 0;
    cudaError_t e = precision == 64 ? launch_typed<double>(a, blocks, threads, st, &kid)
                                    : launch_typed<float>(a, blocks, threads, st, &kid);
    if (kernel) *kernel = kid;
    return e;
}

cudaError_t launch_plain_level(const SweepArgs& a, uint32_t begin, uint32_t end, cudaStream_t st) {
    if (end <= begin) return cudaSuccess;
    unsigned blocks = (end - begin + 255) / 256;
    switch (a.G) {
        case 1: k_plain<1><<<blocks, 256, 0, st>>>(a, begin, end); break;
        case 2: k_plain<2><<<blocks, 256, 0, st>>>(a, begin, end); break;
        case 4: k_plain<4><<<blocks, 256, 0, st>>>(a, begin, end); break;
        default: k_plain<0><<<blocks, 256, 0, st>>>(a, begin, end); break;
    }
    return cudaGetLastError();
}

}  // namespace sw
