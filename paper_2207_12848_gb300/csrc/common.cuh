// Internal declarations shared by the libsweep translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sweep.h"

namespace sw {

// ---------------------------------------------------------------------------------------------
// Face-side encoding. A cell's row of the CSR lists every face it touches ("face sides");
// the record is int4 {nbr, An_x, An_y, An_z} with An = A_f * n_out in FP32 bits,
// n_out pointing out of this cell. nbr:
//   >= 0, bit 30 clear : interior neighbour cell
//   >= 0, bit 30 set   : periodic partner cell (nbr & NBR_MASK)
//   <  0               : box boundary face, ordinal b = -1 - nbr (for the boundary inflow array)
// The FP64 twin {n_out.x, n_out.y, n_out.z, A} reproduces the exact classification sign.
// ---------------------------------------------------------------------------------------------
constexpr int32_t NBR_PERIODIC = 0x40000000;
constexpr int32_t NBR_MASK = 0x3fffffff;
constexpr uint32_t TASK_PAD = 0xffffffffu;
constexpr double FOURPI = 4.0 * 3.14159265358979323846;
// |t32| above this fraction of sum|An_i| fixes sign(t32) == sign(t64) (FP32 rounding of An, Omega and the
// dot product is below 6 * 2^-24 of it); inside the band the sign is recomputed in FP64.
constexpr float BAND_REL = 1.0e-6f;
// inflow sides held in a 128-byte operator line; tasks with more take the geometry path
constexpr int OP_MAX = 14;
// Packed operator: a packet is 32 lanes x 16 bytes (two 8-byte slots per lane); a task holds its
// inflow entries, then its header in the odd slot of its last lane, so at most PK_MAX_IN entries.
constexpr int PK_MAX_IN = 63;
constexpr uint32_t PK_BOUNDARY = 0x80000000u;  // source-index bit of a boundary-face entry
// cell update the packed kernel applies: the balance of scheme (a) or (b), the EXP law, or the
// transposed balance of the adjoint sweep (source scaled by the direction weight)
enum { PK_BALANCE = 0, PK_EXP = 1, PK_TRANSPOSED = 2 };
// forms of the assembled operator
enum { OPF_NONE = 0, OPF_LINES = 1, OPF_PACKETS = 2 };

struct GridBar {
    unsigned count;
    unsigned gen;
};

// FP64 face-side twin {n_out.x, n_out.y, n_out.z, A}, one 32-byte sector
struct alignas(32) d4 {
    double x, y, z, w;
};

// Device error word values (the first error wins).
enum { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_OVERFLOW = 2 };

// ---------------------------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float ld_relaxed(const float* p) {
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ double ld_relaxed(const double* p) {
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
// the G intensities of one cell and direction in one access (each 32-bit element on its own is what
// the readiness test looks at, so the vector needs no atomicity across elements)
__device__ __forceinline__ float2 ld_relaxed_v2(const float* p) {
    float2 v;
    asm volatile("ld.relaxed.gpu.global.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ float4 ld_relaxed_v4(const float* p) {
    float4 v;
    asm volatile("ld.relaxed.gpu.global.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_relaxed_v2(float* p, float2 v) {
    asm volatile("st.relaxed.gpu.global.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v.x), "f"(v.y));
}
__device__ __forceinline__ void st_relaxed_v4(float* p, float4 v) {
    asm volatile("st.relaxed.gpu.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w));
}
// relaxed accesses with an L2 eviction-priority hint (createpolicy), for values read again soon
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ float ld_relaxed_hint(const float* p, uint64_t pol) {
    float v;
    asm volatile("ld.relaxed.gpu.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_relaxed_hint(float* p, float v, uint64_t pol) {
    asm volatile("st.relaxed.gpu.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol));
}
__device__ __forceinline__ float2 ld_relaxed_hint_v2(const float* p, uint64_t pol) {
    float2 v;
    asm volatile("ld.relaxed.gpu.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
                 : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float4 ld_relaxed_hint_v4(const float* p, uint64_t pol) {
    float4 v;
    asm volatile("ld.relaxed.gpu.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_relaxed_hint_v2(float* p, float2 v, uint64_t pol) {
    asm volatile("st.relaxed.gpu.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y),
                 "l"(pol));
}
__device__ __forceinline__ void st_relaxed_hint_v4(float* p, float4 v, uint64_t pol) {
    asm volatile("st.relaxed.gpu.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x),
                 "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol));
}
// Predicated forms (the access is issued only where `on` is set; a load leaves 0 elsewhere): one
// predicated instruction instead of a branch around an asm statement, so lanes of a warp that skip
// the access do not diverge.
__device__ __forceinline__ float ld_relaxed_hint_if(const float* p, uint64_t pol, bool on) {
    float v = 0.f;
    asm volatile("{ .reg .pred q; setp.ne.u32 q, %3, 0; @q ld.relaxed.gpu.global.L2::cache_hint.f32 %0, [%1], %2; }"
                 : "+f"(v) : "l"(p), "l"(pol), "r"((unsigned)on));
    return v;
}
__device__ __forceinline__ float2 ld_relaxed_hint_v2_if(const float* p, uint64_t pol, bool on) {
    float2 v = make_float2(0.f, 0.f);
    asm volatile("{ .reg .pred q; setp.ne.u32 q, %4, 0; @q ld.relaxed.gpu.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3; }"
                 : "+f"(v.x), "+f"(v.y) : "l"(p), "l"(pol), "r"((unsigned)on));
    return v;
}
__device__ __forceinline__ float4 ld_relaxed_hint_v4_if(const float* p, uint64_t pol, bool on) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    asm volatile("{ .reg .pred q; setp.ne.u32 q, %6, 0; @q ld.relaxed.gpu.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5; }"
                 : "+f"(v.x), "+f"(v.y), "+f"(v.z), "+f"(v.w) : "l"(p), "l"(pol), "r"((unsigned)on));
    return v;
}
// predicated re-read that keeps the previous value where `on` is clear
__device__ __forceinline__ float ld_relaxed_keep_if(const float* p, bool on, float old) {
    float v = old;
    asm volatile("{ .reg .pred q; setp.ne.u32 q, %2, 0; @q ld.relaxed.gpu.global.f32 %0, [%1]; }"
                 : "+f"(v) : "l"(p), "r"((unsigned)on));
    return v;
}
__device__ __forceinline__ void ld_relaxed_keep_v2_if(const float* p, bool on, float* x) {
    asm volatile("{ .reg .pred q; setp.ne.u32 q, %3, 0; @q ld.relaxed.gpu.global.v2.f32 {%0, %1}, [%2]; }"
                 : "+f"(x[0]), "+f"(x[1]) : "l"(p), "r"((unsigned)on));
}
__device__ __forceinline__ void ld_relaxed_keep_v4_if(const float* p, bool on, float* x) {
    asm volatile("{ .reg .pred q; setp.ne.u32 q, %5, 0; @q ld.relaxed.gpu.global.v4.f32 {%0, %1, %2, %3}, [%4]; }"
                 : "+f"(x[0]), "+f"(x[1]), "+f"(x[2]), "+f"(x[3]) : "l"(p), "r"((unsigned)on));
}
// read-only data of the launch (not written by the kernel itself)
__device__ __forceinline__ float4 ld_nc_v4_if(const void* p, bool on) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    asm volatile("{ .reg .pred q; setp.ne.u32 q, %5, 0; @q ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4]; }"
                 : "+f"(v.x), "+f"(v.y), "+f"(v.z), "+f"(v.w) : "l"(p), "r"((unsigned)on));
    return v;
}
__device__ __forceinline__ float2 ld_nc_v2_if(const void* p, bool on) {
    float2 v = make_float2(0.f, 0.f);
    asm volatile("{ .reg .pred q; setp.ne.u32 q, %3, 0; @q ld.global.nc.v2.f32 {%0, %1}, [%2]; }"
                 : "+f"(v.x), "+f"(v.y) : "l"(p), "r"((unsigned)on));
    return v;
}
__device__ __forceinline__ void st_relaxed_hint_if(float* p, float v, uint64_t pol, bool on) {
    asm volatile("{ .reg .pred q; setp.ne.u32 q, %3, 0; @q st.relaxed.gpu.global.L2::cache_hint.f32 [%0], %1, %2; }"
                 ::"l"(p), "f"(v), "l"(pol), "r"((unsigned)on));
}
__device__ __forceinline__ void st_relaxed_hint_v2_if(float* p, float2 v, uint64_t pol, bool on) {
    asm volatile("{ .reg .pred q; setp.ne.u32 q, %4, 0; @q st.relaxed.gpu.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3; }"
                 ::"l"(p), "f"(v.x), "f"(v.y), "l"(pol), "r"((unsigned)on));
}
__device__ __forceinline__ void st_relaxed_hint_v4_if(float* p, float4 v, uint64_t pol, bool on) {
    asm volatile("{ .reg .pred q; setp.ne.u32 q, %6, 0; @q st.relaxed.gpu.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5; }"
                 ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol), "r"((unsigned)on));
}
__device__ __forceinline__ void st_relaxed(float* p, float v) {
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v));
}
__device__ __forceinline__ void st_relaxed(double* p, double v) {
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v));
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ void st_relaxed_i32(int* p, int v) {
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// L2 policy that marks lines first in line for eviction (streamed CSR records)
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// streaming read of CSR records: read-only path, no L1 allocation, evict-first in L2
__device__ __forceinline__ int4 ld_stream_int4(const int4* p, uint64_t pol) {
    int4 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ bool sign_bit(float v) { return (__float_as_uint(v) >> 31) != 0; }
__device__ __forceinline__ bool sign_bit(double v) { return (__double_as_longlong(v) >> 63) != 0; }

// Exact FP64 classification value t = ((nx*Ox) + (ny*Oy)) + (nz*Oz), no fused multiply-add
// (the same rounding sequence as the oracle, so signs agree bit for bit).
__device__ __forceinline__ double exact_t(const d4& n, const double* om) {
    double x = __dmul_rn(n.x, om[0]);
    double y = __dmul_rn(n.y, om[1]);
    double z = __dmul_rn(n.z, om[2]);
    return __dadd_rn(__dadd_rn(x, y), z);
}

// FP32 weight of a face side: An.Omega with one fixed rounding sequence (used by every kernel, so the
// two sides of a face get weights of exactly equal magnitude)
__device__ __forceinline__ float dot32(float ax, float ay, float az, const float4& om) {
    return fmaf(az, om.z, fmaf(ay, om.y, __fmul_rn(ax, om.x)));
}

// Classification of one face side for a direction: +1 outflow, -1 inflow, 0 tie (no flux).
// t32 is the FP32 dot product An.Omega; the FP64 twin decides inside the rounding band.
static __device__ __noinline__ int exact_sign(const d4* side64, uint32_t s, const double* om64) {
    const double t = exact_t(side64[s], om64);
    return t > 0.0 ? 1 : (t < 0.0 ? -1 : 0);
}
__device__ __forceinline__ int classify_side(float t32, float ax, float ay, float az, const d4* side64,
                                             uint32_t s, const double* om64) {
    const float band = BAND_REL * (fabsf(ax) + fabsf(ay) + fabsf(az));
    if (t32 > band) return 1;
    if (t32 < -band) return -1;
    return exact_sign(side64, s, om64);
}

// FP32 weight |a.Omega| of a face side (a = A n_out, its area vector), accurate to about one
// rounding for every side, grazing ones included. The area vector and the direction are each
// carried as an FP32 pair hi + lo (hi in the side record and the FP32 direction, lo beside them);
// the hi-hi products are formed exactly (product plus its FMA residual) and summed with
// error-free two-sums, and the residuals and hi-lo cross terms are added as one correction. Every
// step is symmetric under negation, so the two sides of a face (exactly negated records) get
// weights of exactly equal magnitude.
__device__ __forceinline__ float dot_comp(float ax, float ay, float az, const float4& lo, const float4& om,
                                          const float4& oml) {
    const float px = __fmul_rn(ax, om.x), py = __fmul_rn(ay, om.y), pz = __fmul_rn(az, om.z);
    const float ex = fmaf(ax, om.x, -px), ey = fmaf(ay, om.y, -py), ez = fmaf(az, om.z, -pz);
    const float s1 = __fadd_rn(px, py);
    const float b1 = __fsub_rn(s1, px);
    const float r1 = __fadd_rn(__fsub_rn(px, __fsub_rn(s1, b1)), __fsub_rn(py, b1));
    const float s2 = __fadd_rn(s1, pz);
    const float b2 = __fsub_rn(s2, s1);
    const float r2 = __fadd_rn(__fsub_rn(s1, __fsub_rn(s2, b2)), __fsub_rn(pz, b2));
    float c = __fadd_rn(__fadd_rn(__fadd_rn(ex, ey), ez), __fadd_rn(r1, r2));
    c = fmaf(ax, oml.x, c);
    c = fmaf(ay, oml.y, c);
    c = fmaf(az, oml.z, c);
    c = fmaf(lo.x, om.x, c);
    c = fmaf(lo.y, om.y, c);
    c = fmaf(lo.z, om.z, c);
    return __fadd_rn(s2, c);
}

__device__ __forceinline__ float side_weight(const int4& r, const float4& lo, const float4& om, const float4& oml) {
    return fabsf(dot_comp(__int_as_float(r.y), __int_as_float(r.z), __int_as_float(r.w), lo, om, oml));
}

// Grid-wide barrier for persistent cooperative kernels, with a bounded wait.
// Returns false (and sets *err) if the wait gave up or another block reported an error.
__device__ __forceinline__ bool grid_sync(GridBar* bar, unsigned nblocks, long long budget, int* err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned gen = ld_acquire_u32(&bar->gen);
        __threadfence();
        unsigned arrived = atomicAdd(&bar->count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            st_release_u32(&bar->gen, gen + 1);
        } else {
            long long n = 0;
            while (ld_acquire_u32(&bar->gen) == gen) {
                if (++n > budget || ld_volatile_i32(err) != DEV_OK) {
                    atomicCAS(err, DEV_OK, DEV_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (ld_volatile_i32(err) != DEV_OK) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------------------------------------
// Host-side structures
// ---------------------------------------------------------------------------------------------
struct DevMesh {
    int64_t N = 0, F = 0, S = 0, NB = 0;  // cells, faces, face sides, boundary faces
    uint32_t* rowptr = nullptr;            // [N+1]
    int4* side = nullptr;                  // [S]
    d4* side64 = nullptr;                  // [S]
    float4* side_lo = nullptr;             // [S] area vector minus its FP32 value in the side record
    int2* nbr_rows = nullptr;              // [S] row bounds of the side's interior neighbour ({0, 0} otherwise)
    uint32_t* twin = nullptr;              // [S] position of the same face in the neighbour's row (interior and
                                           //     periodic sides; boundary sides 0xffffffff)
    double* vol = nullptr;                 // [N]
    int32_t* pcells = nullptr;             // cells with periodic sides
    int64_t n_pcells = 0;
    int32_t* bcells = nullptr;             // cells with boundary sides
    int64_t n_bcells = 0;
    int max_row = 0;
    std::vector<int64_t> mesh_off;
};

// A packed operator: packets of 32 int4 with their {head mask, long-task flag}, the first packet of
// each level of its stream, and the packing groups (runs of up to 32 chunks of one level) with their
// packet counts. The forward operator streams the levels in sweep order, the transposed one in reverse.
struct PackedOp {
    int4* pk = nullptr;
    uint2* meta = nullptr;
    int64_t cap = 0;             // packets allocated
    int64_t n_pk = 0;            // packets of the current operator (even within every level)
    int64_t* lev_pk = nullptr;   // device [n_levels+1] first packet of each level of the stream
    int2* grp = nullptr;         // device [ng] {first chunk, end chunk} of each packing group
    int32_t* lev_grp = nullptr;  // device [n_levels+1] first group of each level of the stream
    int32_t* cnt = nullptr;      // device [ng] packets per group
    int64_t* off = nullptr;      // device [ng+1] first packet of each group
    int64_t* scan = nullptr;     // scan scratch
    int64_t grp_cap = 0;         // groups (and levels + 1) the tables above hold
    int64_t ng = 0;
    int32_t* flag = nullptr;     // device word: a task has more entries than a packet holds
    bool valid = false;          // transposed operator: built for the current levels
};

struct Levels {
    bool valid = false;
    int d0 = 0, nd = 0;
    int cshift = 0;
    uint32_t cmask = 0;
    int n_levels = 0;
    uint32_t* raw = nullptr;     // level-contiguous, padded task list written by the levelisation
    uint32_t* task = nullptr;    // same levels, grouped by direction within each level
    int64_t task_cap = 0;
    int4* info = nullptr;        // [N][nd] {upwind count, P_c (FP32), inflow mask, outflow mask}
    int4* trec = nullptr;        // task records {entry, row start, P_c, inflow mask}, same order as task
    int4* op = nullptr;          // assembled operator: headers then entries (see build_operator), or null
    size_t op_bytes = 0;
    bool op_valid = false;
    int op_format = OPF_NONE;    // form of the assembled operator when op_valid
    PackedOp pk;                 // packed operator of the forward sweep (OPF_PACKETS)
    PackedOp pkt;                // packed transposed operator of the adjoint sweep, built on demand
    // direction-conserving transport (scheme (b) of Sec. 2.6), [N][nd] like info: the chosen outflow
    // sides (bit k = row position k), the effective inflow sides (interior and periodic sides the
    // upwind cell chose, boundary inflow sides), and the share P_c / n_c each chosen side carries
    int transport = 0;           // 0 = scheme (a); n = scheme (b) to n neighbours
    uint64_t* dc_mask = nullptr;
    uint64_t* dc_inm = nullptr;
    float* dc_share32 = nullptr;
    double* dc_share64 = nullptr;
    int32_t* level = nullptr;    // [nd][N] (during levelisation: minus the upwind cells still unsolved)
    int32_t* lvl_cnt = nullptr;  // [N+2]
    uint32_t* pad_off = nullptr; // [N+2] start of each level in the padded list
    int64_t* lev_chunk = nullptr;  // device [n_levels+1] chunk (32-task) offsets
    uint32_t* seg_off = nullptr; // device [n_levels][nd+1] per-(level, direction) segment starts
    int64_t seg_cap = 0;         // elements allocated for seg_off
    std::vector<int64_t> h_lev_chunk;
    std::vector<uint32_t> h_seg_off;
    std::vector<int32_t> depth;  // per direction
    int64_t n_tasks = 0;
    // direction-parallel levelisation: per direction, the cells per level and the start of each level
    // in that direction's list, for up to dlev_cap levels; then level-0 sizes, depths, overflow word
    int32_t* dlev = nullptr;     // [nd][2][dlev_cap] + [nd] + [nd] + [1]
    int dlev_cap = 0;
    int32_t* lfill = nullptr;    // [nd][dlev_cap] positions taken within each level while ordering the lists
};

// Kernel argument block of the batched sweep.
struct SweepArgs {
    const uint32_t* task;
    const int4* trec;     // task records (FP32 forward sweep)
    const int4* op;       // assembled operator headers (one int4 per task), or null (FP32 forward sweep)
    const int4* pk;       // packed operator (FP32 forward sweep), or null
    // scheme (b): per [N][nd] chosen outflow sides and shares, per side the twin's row position (null: scheme (a))
    const uint64_t* dc_mask;
    const float* dc_share32;
    const double* dc_share64;
    const uint32_t* twin;
    const uint2* pk_meta; // [n_pk] {head mask, long-task flag} of each packet
    int64_t n_pk;
    const int64_t* lev_pk;  // [n_levels+1] first packet of each level
    int64_t n_chunks;
    const int64_t* lev_chunk;
    int n_levels;
    int cshift;
    uint32_t cmask;
    int nd;               // directions of this batch
    const uint32_t* rowptr;
    const int4* side;
    const d4* side64;
    const float4* side_lo;  // [S] low parts of the area vectors
    const float4* om32;   // [nd]
    const float4* om32lo; // [nd] low parts of the directions
    const double* om64;   // [nd][3]
    const double* w64;    // [nd] weights (adjoint source scaling)
    const void* cm;       // [N][G] {q, dnm} in the sweep precision
    const void* bc;       // [NB][G] boundary inflow, or null
    void* I;              // [nd][N][G] output
    const void* Iprev;    // [nd][N][G] previous sweep (periodic inflow), or null
    int64_t N;
    int G;
    int parity;           // sign bit written with every value of this sweep
    int reverse;          // 1 = adjoint (transposed) sweep
    int level_sync;       // 1 = grid barrier between levels
    int lanes;            // lanes cooperating on one task (4 or 8) in the batched kernel
    int law;              // 0 = BALANCE, 1 = EXP (forward sweeps of the generic and plain kernels)
    void* Imean;          // EXP: [nd][N][G] cell-mean intensity written by the sweep
    GridBar* bar;
    int* err;
    long long spin_budget;
    int debug_stall;
    const float* stall_word;
};

// ---------------------------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files)
// ---------------------------------------------------------------------------------------------
cudaError_t launch_build_csr(const DevMesh& m, const int32_t* d_fc, const double* d_area, const double* d_normal,
                             const uint8_t* d_flags, int32_t* d_tmp_cnt, cudaStream_t st);
cudaError_t launch_validate_mesh(int64_t N, int64_t F, const double* vol, const int32_t* fc, const double* area,
                                 const double* normal, const uint8_t* flags, const int64_t* mesh_off, int n_meshes,
                                 int* d_bad, cudaStream_t st);

cudaError_t build_operator(const DevMesh& m, const Levels& L, const double* om64_all, const float4* om32_all,
                           const float4* om32lo_all, cudaStream_t st);
// packed operator P of the levels L: plan (groups, packet counts; *n_pk = packets needed, or -1 when a
// task has more entries than a packet holds) then write into P.pk / P.meta. transposed: the adjoint's
// operator (outflow entries, levels in reverse order)
cudaError_t pack_plan(const DevMesh& m, const Levels& L, PackedOp& P, bool transposed, const double* om64_all,
                      const float4* om32_all, const float4* om32lo_all, cudaStream_t st, int64_t* n_pk);
cudaError_t pack_write(const DevMesh& m, const Levels& L, PackedOp& P, bool transposed, const double* om64_all,
                       const float4* om32_all, const float4* om32lo_all, cudaStream_t st);
cudaError_t levelise(const DevMesh& m, Levels& L, const double* om64_all, const float4* om32_all,
                     const float4* om32lo_all, int dev_sms, GridBar* bar, int* err, long long budget,
                     int64_t* d_scratch, cudaStream_t st, float* t_classify, float* t_levelise, std::string* msg);

// fmt: OPF_* form of the assembled operator the launch reads (OPF_NONE: the mesh rows); generic: the
// mesh-row launch is the generic kernel (reverse, EXP, scheme (b)); pk_mode: the packed kernel's PK_*
int sweep_occupancy(int precision, int G, int threads, int nd, int lanes, int generic, int fmt, int pk_mode);
cudaError_t launch_sweep(const SweepArgs& a, int precision, int blocks, int threads, cudaStream_t st,
                         int* kernel = nullptr);
cudaError_t launch_plain_level(const SweepArgs& a, uint32_t begin, uint32_t end, cudaStream_t st);

cudaError_t launch_prep_material(int64_t N, int G, const double* vol, const double* ka, const double* ks,
                                 const double* em, const double* J, float2* cm32, double2* cm64, cudaStream_t st);
cudaError_t launch_prep_adjoint_src(int64_t N, int G, const double* vol, const double* ka, const double* ks,
                                    const double* dl_dJ, const double* dl_dG, float2* cm32, double2* cm64,
                                    cudaStream_t st);
cudaError_t launch_tally(int precision, const void* I, int64_t N, int G, int nd, int d0, const double* w64,
                         double wsum, const double* vol, const double* ka, const double* em, double* J,
                         double* Gam, double* partial, int nblk, cudaStream_t st);
// scheme (b) tables of a solve ([N][nd] chosen outflow sides and FP64 shares, per side the twin's row
// position); a null pointer to it, or a null mask, means scheme (a)
struct DcTabs {
    const uint64_t* mask = nullptr;
    const double* share64 = nullptr;
    const uint32_t* twin = nullptr;
};
cudaError_t launch_boundary_tally(int precision, const DevMesh& m, const void* I, int G, int nd, int d0,
                                  const double* om64, const double* w64, const double* bc, double* partial,
                                  int nblk, cudaStream_t st, const DcTabs* dc = nullptr);
cudaError_t launch_scat_residual(int64_t NG, const double* J, double* Jold, unsigned long long* d_max,
                                 cudaStream_t st);
// FP64 periodic-inflow weights of a solve (periodic sides of the periodic cells x directions)
struct PeriodicTable {
    int32_t* off = nullptr;   // [n_pcells+1] first periodic side of each periodic cell, then scratch counts
    size_t off_cap = 0;
    double* wa = nullptr;     // [periodic sides][nd] w_d A |n.Omega| on inflow sides, else 0
    size_t wa_cap = 0;
    bool ready = false;
};
cudaError_t build_periodic_table(const DevMesh& m, int nd, const double* om64, const double* w64, PeriodicTable* t,
                                 cudaStream_t st, const DcTabs* dc = nullptr);
cudaError_t launch_periodic_source(int precision, const DevMesh& m, const void* I, int G, int nd,
                                   const double* om64, const double* w64, double* jn1, const double* jn,
                                   unsigned long long* d_max, double* partial, int nblk, cudaStream_t st,
                                   const PeriodicTable* tab = nullptr);
cudaError_t launch_reduce_sum(const double* partial, int n, double* out, cudaStream_t st);
cudaError_t launch_grad_accum(int precision, const void* I, const void* lam, int64_t N, int G, int nd, int d0,
                              const double* w64, const double* vol, const double* dl_dG, double* gk, double* ge,
                              cudaStream_t st);
cudaError_t launch_fill_u32(uint32_t* p, uint32_t v, int64_t n, cudaStream_t st);
// rotation of the direction set: quadrature counts of the shared bins, and the remap of [D][NG] intensities
cudaError_t launch_remap_count(const double3* pts, int64_t n, const double* om_old, const double* om_new, int n_dir,
                               unsigned long long* cnt, cudaStream_t st);
cudaError_t launch_remap(int precision, const void* in, void* out, int64_t NG, int n_dir, const int32_t* rp,
                         const int32_t* col, const double* val, int par, cudaStream_t st);
cudaError_t launch_to_f64(int precision, const void* I, int64_t n, double* out, cudaStream_t st);

}  // namespace sw
