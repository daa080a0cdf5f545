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
//   LEVEL    -- warps take 32-task chunks of one wavefront level round-robin; grid barrier per level.
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
__device__ __forceinline__ float divr(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double divr(double a, double b) { return __ddiv_rn(a, b); }

// Wait (bounded) until *p carries this sweep's parity; returns the magnitude. false on give-up.
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

// One task (c, Omega) for all groups. GC = compile-time group count (0: runtime a.G <= 8).
template <typename real, int GC>
__device__ __forceinline__ bool run_task(const SweepArgs& a, uint32_t entry, const float4* s_om, bool stall) {
    constexpr bool F64 = sizeof(real) == 8;
    constexpr int GM = GC > 0 ? GC : 8;
    const int G = GC > 0 ? GC : a.G;
    using real2 = typename vec2<real>::type;
    const uint32_t c = entry & a.cmask;
    const uint32_t dl = entry >> a.cshift;
    const uint32_t r0 = __ldg(a.rowptr + c), r1 = __ldg(a.rowptr + c + 1);
    const double* om64 = a.om64 + 3 * dl;
    const float4 om = F64 ? make_float4(0.f, 0.f, 0.f, 0.f) : s_om[dl];
    const real2* cm = reinterpret_cast<const real2*>(a.cm) + (size_t)c * G;
    real acc[GM], dnm[GM];
    const real wsc = a.reverse ? (real)a.w64[dl] : (real)1;
#pragma unroll
    for (int g = 0; g < GM; ++g) {
        if (g < G) {
            real2 v = cm[g];
            acc[g] = a.reverse ? mulr(wsc, v.x) : v.x;
            dnm[g] = v.y;
        }
    }
    if (stall) {  // test hook: wait on a word that nothing writes
        real dummy;
        if (!wait_value(reinterpret_cast<const real*>(a.stall_word), 1, a, dummy)) return false;
    }
    real P = 0;
    real* I = reinterpret_cast<real*>(a.I);
    const size_t slab = (size_t)dl * a.N;
    const uint64_t pol = policy_evict_first();
    for (uint32_t s = r0; s < r1; ++s) {
        const int4 rec = ld_stream_int4(a.side + s, pol);
        real w;
        int sgn;
        if (F64) {
            const d4 n = a.side64[s];
            const double t = exact_t(n, om64);
            sgn = t > 0.0 ? 1 : (t < 0.0 ? -1 : 0);
            w = (real)__dmul_rn(n.w, fabs(t));
        } else {
            const float ax = __int_as_float(rec.y), ay = __int_as_float(rec.z), az = __int_as_float(rec.w);
            const float t32 = fmaf(az, om.z, fmaf(ay, om.y, ax * om.x));
            sgn = classify_side(t32, ax, ay, az, a.side64, s, om64);
            w = (real)fabsf(t32);
        }
        if (sgn == 0) continue;
        if (sgn > 0) P = addr(P, w);
        const bool inflow = a.reverse ? (sgn > 0) : (sgn < 0);
        if (!inflow) continue;
        const int32_t nb = rec.x;
        if (nb >= 0 && !(nb & NBR_PERIODIC)) {
            const real* src = I + (slab + (uint32_t)nb) * G;
#pragma unroll
            for (int g = 0; g < GM; ++g) {
                if (g < G) {
                    real v;
                    if (!wait_value(src + g, a.parity, a, v)) return false;
                    acc[g] = fmar(w, v, acc[g]);
                }
            }
        } else if (a.reverse) {
            // the adjoint has no boundary or periodic source
        } else if (nb >= 0) {
            if (a.Iprev) {
                const real* src = reinterpret_cast<const real*>(a.Iprev) + (slab + (uint32_t)(nb & NBR_MASK)) * G;
#pragma unroll
                for (int g = 0; g < GM; ++g)
                    if (g < G) acc[g] = fmar(w, (real)fabs(src[g]), acc[g]);
            }
        } else if (a.bc) {
            const real* b = reinterpret_cast<const real*>(a.bc) + (size_t)(-1 - nb) * G;
#pragma unroll
            for (int g = 0; g < GM; ++g)
                if (g < G) acc[g] = fmar(w, b[g], acc[g]);
        }
    }
    real* dst = I + (slab + c) * G;
#pragma unroll
    for (int g = 0; g < GM; ++g) {
        if (g < G) {
            real v = divr(acc[g], addr(P, dnm[g]));
            st_relaxed(dst + g, a.parity ? -v : v);
        }
    }
    return true;
}

template <typename real, int GC>
__global__ void __launch_bounds__(256) k_sweep(SweepArgs a) {
    extern __shared__ float4 s_om[];
    for (int i = threadIdx.x; i < a.nd; i += blockDim.x) s_om[i] = a.om32[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (a.level_sync) {
        bool ok = true;
        for (int li = 0; li < a.n_levels; ++li) {
            const int L = a.reverse ? a.n_levels - 1 - li : li;
            const int64_t k0 = a.lev_chunk[L], k1 = a.lev_chunk[L + 1];
            if (ok) {
                for (int64_t k = k0 + warp; k < k1; k += nwarps) {
                    const uint32_t e = a.task[k * 32 + lane];
                    if (e != TASK_PAD) {
                        const bool stall = a.debug_stall && k == 0 && lane == 0;
                        if (!run_task<real, GC>(a, e, s_om, stall)) { ok = false; break; }
                    }
                }
            }
            if (!grid_sync(a.bar, gridDim.x, a.spin_budget, a.err)) return;
        }
    } else {
        for (int64_t i = 0;; ++i) {
            const int64_t k = a.reverse ? (a.n_chunks - 1 - warp - i * nwarps) : (warp + i * nwarps);
            if (k < 0 || k >= a.n_chunks) break;
            if ((i & 7) == 0 && ld_volatile_i32(a.err) != DEV_OK) return;
            const uint32_t e = a.task[k * 32 + lane];
            if (e != TASK_PAD) {
                const bool stall = a.debug_stall && i == 0 && warp == 0 && lane == 0;
                if (!run_task<real, GC>(a, e, s_om, stall)) return;
            }
        }
    }
}

// K8: the plain path -- one launch per (direction, level) segment, FP64, thread per task.
template <int GC>
__global__ void __launch_bounds__(256) k_plain(SweepArgs a, uint32_t begin, uint32_t end) {
    const uint32_t i = begin + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= end) return;
    run_task<double, GC>(a, a.task[i], nullptr, false);
}

template <typename real>
cudaError_t launch_typed(const SweepArgs& a, int blocks, int threads, cudaStream_t st) {
    size_t smem = sizeof(float4) * (size_t)a.nd;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    switch (a.G) {
        case 1: return cudaLaunchKernelEx(&cfg, k_sweep<real, 1>, a);
        case 2: return cudaLaunchKernelEx(&cfg, k_sweep<real, 2>, a);
        case 4: return cudaLaunchKernelEx(&cfg, k_sweep<real, 4>, a);
        default: return cudaLaunchKernelEx(&cfg, k_sweep<real, 0>, a);
    }
}

template <typename real>
int occupancy_typed(int G, int threads, size_t smem) {
    int n = 0;
    switch (G) {
        case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<real, 1>, threads, smem); break;
        case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<real, 2>, threads, smem); break;
        case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<real, 4>, threads, smem); break;
        default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<real, 0>, threads, smem); break;
    }
    return n;
}

}  // namespace

int sweep_occupancy(int precision, int G, int threads, int nd) {
    size_t smem = sizeof(float4) * (size_t)nd;
    return precision == 64 ? occupancy_typed<double>(G, threads, smem) : occupancy_typed<float>(G, threads, smem);
}

int sweep_max_blocks_per_sm(int precision, int threads) { return sweep_occupancy(precision, 1, threads, 1024); }

cudaError_t launch_sweep(const SweepArgs& a, int precision, int blocks, int threads, cudaStream_t st) {
    return precision == 64 ? launch_typed<double>(a, blocks, threads, st) : launch_typed<float>(a, blocks, threads, st);
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
