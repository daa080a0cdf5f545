// Mesh upload, CSR build, face classification (K1) and GPU Kahn levelisation (K2).
//
// Classification: a neighbour across face side s is downwind when n_out.Omega > 0 and upwind
// when < 0 (paper Sec. 2.5 and Appendix A, Eq. downwindDefinition); an exact FP64 zero carries
// no flux and creates no dependency. Periodic and boundary sides create no dependency
// (the periodic graph is cut, Sec. 2.7).
//
// Levelisation: the level of a task (c, Omega) is 0 when it has no upwind cell, else
// 1 + the largest level of its upwind cells -- the longest dependency path, which is unique
// for an acyclic graph (Sec. 2.3). K2 is Alg. 2's Kahn queue run one wavefront at a time for
// all directions at once: the tasks of level L decrement the upwind counters n(c, Omega) of
// their downwind neighbours; a counter reaching zero puts that task into level L+1.
#include <algorithm>
#include <cooperative_groups.h>

#include "common.cuh"

namespace sw {

namespace {

constexpr int SCAN_BLOCK = 1024;
constexpr int SCAN_ITEMS = 4;

// ---- exclusive scan (int32 counts -> int64 offsets), three passes ----------------------------
__global__ void k_scan_block(const int32_t* in, int64_t n, int64_t* out, int64_t* block_sums) {
    __shared__ int64_t s[SCAN_BLOCK];
    int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t sum = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
        v[k] = i < n ? (int64_t)in[i] : 0;
        sum += v[k];
    }
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
        int64_t t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    int64_t run = s[threadIdx.x] - sum;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    if (threadIdx.x == SCAN_BLOCK - 1) block_sums[blockIdx.x] = s[threadIdx.x];
}

__global__ void k_scan_sums(int64_t* sums, int64_t nb, int64_t* total) {
    // one block, sequential chunks of SCAN_BLOCK
    __shared__ int64_t s[SCAN_BLOCK];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nb; b0 += SCAN_BLOCK) {
        int64_t i = b0 + threadIdx.x;
        int64_t v = i < nb ? sums[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
            int64_t t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) sums[i] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == SCAN_BLOCK - 1) carry += s[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int64_t* out, int64_t n, const int64_t* sums) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += sums[i / (SCAN_BLOCK * SCAN_ITEMS)];
}

// exclusive scan of n int32 into out[n] (int64); total at out_total (device). scratch >= nblocks+1
cudaError_t scan_i32(const int32_t* in, int64_t n, int64_t* out, int64_t* scratch, int64_t* out_total,
                     cudaStream_t st) {
    int64_t per = (int64_t)SCAN_BLOCK * SCAN_ITEMS;
    int64_t nb = (n + per - 1) / per;
    if (nb == 0) nb = 1;
    k_scan_block<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(in, n, out, scratch);
    k_scan_sums<<<1, SCAN_BLOCK, 0, st>>>(scratch, nb, out_total);
    if (n > 0) k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n, scratch);
    return cudaGetLastError();
}

// ---- mesh validation -------------------------------------------------------------------------
enum {
    BAD_CELL_RANGE = 1, BAD_FLAGS = 2, BAD_AREA = 4, BAD_NORMAL = 8, BAD_VOLUME = 16, BAD_CROSS_MESH = 32,
    BAD_SELF = 64
};

__device__ int64_t mesh_of(const int64_t* off, int nm, int64_t c) {
    int lo = 0, hi = nm;  // off[lo] <= c < off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= c) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void k_validate_faces(int64_t N, int64_t F, const int32_t* fc, const double* area, const double* normal,
                                 const uint8_t* flags, const int64_t* mesh_off, int nm, int* bad) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    int b = 0;
    int32_t c0 = fc[2 * f], c1 = fc[2 * f + 1];
    uint8_t fl = flags[f];
    if (c0 < 0 || c0 >= N || c1 < -1 || c1 >= N) b |= BAD_CELL_RANGE;
    bool bnd = (fl & SWEEP_FACE_BOUNDARY) != 0, per = (fl & SWEEP_FACE_PERIODIC) != 0;
    if ((fl & ~3) || (bnd && per) || (bnd != (c1 == -1))) b |= BAD_FLAGS;
    if (c0 == c1 && !per) b |= BAD_SELF;
    double A = area[f];
    if (!(A >= 0.0) || !isfinite(A)) b |= BAD_AREA;
    double nx = normal[3 * f], ny = normal[3 * f + 1], nz = normal[3 * f + 2];
    double n2 = nx * nx + ny * ny + nz * nz;
    if (!(fabs(n2 - 1.0) <= 2.5e-9)) b |= BAD_NORMAL;
    if (!b && c1 >= 0 && nm > 1 && mesh_of(mesh_off, nm, c0) != mesh_of(mesh_off, nm, c1)) b |= BAD_CROSS_MESH;
    if (b) atomicOr(bad, b);
}

__global__ void k_validate_cells(int64_t N, const double* vol, int* bad) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    double v = vol[c];
    if (!(v > 0.0) || !isfinite(v)) atomicOr(bad, BAD_VOLUME);
}

// ---- CSR build --------------------------------------------------------------------------------
__global__ void k_count_sides(int64_t F, const int32_t* fc, int32_t* cnt) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    atomicAdd(&cnt[fc[2 * f]], 1);
    if (fc[2 * f + 1] >= 0) atomicAdd(&cnt[fc[2 * f + 1]], 1);
}

__global__ void k_to_u32(const int64_t* in, int64_t n, uint32_t* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (uint32_t)in[i];
}

__global__ void k_scatter_sides(int64_t F, const int32_t* fc, const uint32_t* rowptr, int32_t* fill, int64_t* key) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    int32_t c0 = fc[2 * f], c1 = fc[2 * f + 1];
    uint32_t s0 = rowptr[c0] + atomicAdd(&fill[c0], 1);
    key[s0] = 2 * f;
    if (c1 >= 0) {
        uint32_t s1 = rowptr[c1] + atomicAdd(&fill[c1], 1);
        key[s1] = 2 * f + 1;
    }
}

// rows are short: insertion sort of each row by (face, side) makes the side order deterministic
__global__ void k_sort_rows(int64_t N, const uint32_t* rowptr, int64_t* key, int* max_row) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    uint32_t r0 = rowptr[c], r1 = rowptr[c + 1];
    for (uint32_t i = r0 + 1; i < r1; ++i) {
        int64_t k = key[i];
        uint32_t j = i;
        while (j > r0 && key[j - 1] > k) {
            key[j] = key[j - 1];
            --j;
        }
        key[j] = k;
    }
    atomicMax(max_row, (int)(r1 - r0));
}

__global__ void k_flag_boundary(int64_t F, const uint8_t* flags, int32_t* isb) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f < F) isb[f] = (flags[f] & SWEEP_FACE_BOUNDARY) ? 1 : 0;
}

__global__ void k_fill_sides(int64_t S, const int64_t* key, const int32_t* fc, const double* area,
                             const double* normal, const uint8_t* flags, const int64_t* bidx,
                             const uint32_t* rowptr, int4* side, d4* side64, float4* side_lo, int2* nbr_rows) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    int64_t k = key[s];
    int64_t f = k >> 1;
    int sd = (int)(k & 1);  // 0: this cell is c0 (n_out = n), 1: this cell is c1 (n_out = -n)
    double A = area[f];
    double nx = normal[3 * f], ny = normal[3 * f + 1], nz = normal[3 * f + 2];
    if (sd) { nx = -nx; ny = -ny; nz = -nz; }
    int32_t nbr;
    uint8_t fl = flags[f];
    if (fl & SWEEP_FACE_BOUNDARY) nbr = (int32_t)(-1 - bidx[f]);
    else {
        int32_t other = sd ? fc[2 * f] : fc[2 * f + 1];
        nbr = (fl & SWEEP_FACE_PERIODIC) ? (other | NBR_PERIODIC) : other;
    }
    // area vector A n_out in FP64, as an FP32 value plus its (exactly representable) remainder
    const double ax = A * nx, ay = A * ny, az = A * nz;
    const float hx = (float)ax, hy = (float)ay, hz = (float)az;
    int4 r;
    r.x = nbr;
    r.y = __float_as_int(hx);
    r.z = __float_as_int(hy);
    r.w = __float_as_int(hz);
    side[s] = r;
    side64[s] = d4{nx, ny, nz, A};
    side_lo[s] = make_float4((float)(ax - (double)hx), (float)(ay - (double)hy), (float)(az - (double)hz), 0.f);
    nbr_rows[s] = nbr >= 0 && !(nbr & NBR_PERIODIC) ? make_int2((int)rowptr[nbr], (int)rowptr[nbr + 1]) : make_int2(0, 0);
}

// Position of each interior or periodic side's twin (the same face seen from the neighbour) in the
// neighbour's row: rows are sorted by (face, side), so the twin's key is this key with its side bit
// flipped, found by binary search. Boundary sides get 0xffffffff.
__global__ void k_twin(int64_t S, const int64_t* key, const int32_t* fc, const uint8_t* flags, const uint32_t* rowptr,
                       uint32_t* twin) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int64_t k = key[s], f = k >> 1;
    if (flags[f] & SWEEP_FACE_BOUNDARY) {
        twin[s] = 0xffffffffu;
        return;
    }
    const int32_t u = (k & 1) ? fc[2 * f] : fc[2 * f + 1];
    const int64_t want = k ^ 1;
    uint32_t lo = rowptr[u], hi = rowptr[u + 1];  // key[lo..hi) ascending
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (key[mid] <= want) lo = mid;
        else hi = mid;
    }
    twin[s] = lo - rowptr[u];
}

__global__ void k_cell_kinds(int64_t N, const uint32_t* rowptr, const int4* side, int32_t* isp, int32_t* isb) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    int p = 0, b = 0;
    for (uint32_t s = rowptr[c]; s < rowptr[c + 1]; ++s) {
        int32_t nb = side[s].x;
        if (nb < 0) b = 1;
        else if (nb & NBR_PERIODIC) p = 1;
    }
    isp[c] = p;
    isb[c] = b;
}

__global__ void k_compact(int64_t N, const int32_t* flag, const int64_t* pos, int32_t* out) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N && flag[c]) out[pos[c]] = (int32_t)c;
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_validate_mesh(int64_t N, int64_t F, const double* vol, const int32_t* fc, const double* area,
                                 const double* normal, const uint8_t* flags, const int64_t* mesh_off, int n_meshes,
                                 int* d_bad, cudaStream_t st) {
    if (F > 0) k_validate_faces<<<nblk(F), 256, 0, st>>>(N, F, fc, area, normal, flags, mesh_off, n_meshes, d_bad);
    if (N > 0) k_validate_cells<<<nblk(N), 256, 0, st>>>(N, vol, d_bad);
    return cudaGetLastError();
}

// Builds rowptr/side/side64 and the periodic/boundary cell lists of m (arrays already allocated
// for m.S sides; m.rowptr for N+1). d_tmp_cnt: int32 scratch of max(N, F) + 1.
cudaError_t launch_build_csr(const DevMesh& mc, const int32_t* fc, const double* area, const double* normal,
                             const uint8_t* flags, int32_t* d_tmp, cudaStream_t st) {
    DevMesh& m = const_cast<DevMesh&>(mc);
    int64_t N = m.N, F = m.F, S = m.S;
    cudaError_t e;
    int64_t *off = nullptr, *offb = nullptr, *scratch = nullptr, *key = nullptr, *total = nullptr, *bidx = nullptr;
    int32_t *fill = nullptr, *isp = nullptr, *isb = nullptr;
    int* maxrow = nullptr;
    int64_t nmax = (N > F ? N : F) + 1;
    int64_t nsb = nmax / (SCAN_BLOCK * SCAN_ITEMS) + 2;
#define TRY(x) do { e = (x); if (e != cudaSuccess) goto done; } while (0)
    TRY(cudaMallocAsync(&off, sizeof(int64_t) * (nmax + 1), st));
    TRY(cudaMallocAsync(&offb, sizeof(int64_t) * (N + 1), st));
    TRY(cudaMallocAsync(&scratch, sizeof(int64_t) * nsb, st));
    TRY(cudaMallocAsync(&total, sizeof(int64_t) * 2, st));
    TRY(cudaMallocAsync(&key, sizeof(int64_t) * (S > 0 ? S : 1), st));
    TRY(cudaMallocAsync(&bidx, sizeof(int64_t) * (F + 1), st));
    TRY(cudaMallocAsync(&fill, sizeof(int32_t) * (N + 1), st));
    TRY(cudaMallocAsync(&isp, sizeof(int32_t) * (N + 1), st));
    TRY(cudaMallocAsync(&isb, sizeof(int32_t) * (nmax), st));
    TRY(cudaMallocAsync(&maxrow, sizeof(int), st));
    TRY(cudaMemsetAsync(d_tmp, 0, sizeof(int32_t) * (N + 1), st));
    TRY(cudaMemsetAsync(fill, 0, sizeof(int32_t) * (N + 1), st));
    TRY(cudaMemsetAsync(maxrow, 0, sizeof(int), st));
    if (F > 0) k_count_sides<<<nblk(F), 256, 0, st>>>(F, fc, d_tmp);
    TRY(scan_i32(d_tmp, N + 1, off, scratch, total, st));  // d_tmp[N] = 0 -> off[N] = S
    k_to_u32<<<nblk(N + 1), 256, 0, st>>>(off, N + 1, m.rowptr);
    if (F > 0) k_scatter_sides<<<nblk(F), 256, 0, st>>>(F, fc, m.rowptr, fill, key);
    if (N > 0) k_sort_rows<<<nblk(N, 128), 128, 0, st>>>(N, m.rowptr, key, maxrow);
    // boundary ordinals in face order
    if (F > 0) {
        k_flag_boundary<<<nblk(F), 256, 0, st>>>(F, flags, isb);
        TRY(scan_i32(isb, F, bidx, scratch, total, st));
    }
    if (S > 0) k_fill_sides<<<nblk(S), 256, 0, st>>>(S, key, fc, area, normal, flags, bidx, m.rowptr, m.side,
                                                     m.side64, m.side_lo, m.nbr_rows);
    if (S > 0) k_twin<<<nblk(S), 256, 0, st>>>(S, key, fc, flags, m.rowptr, m.twin);
    // periodic / boundary cell lists (increasing cell order)
    if (N > 0) {
        k_cell_kinds<<<nblk(N), 256, 0, st>>>(N, m.rowptr, m.side, isp, isb);
        TRY(scan_i32(isp, N, off, scratch, total, st));
        TRY(scan_i32(isb, N, offb, scratch, total + 1, st));
    }
    {
        int64_t tot[2] = {0, 0};
        int mr = 0;
        TRY(cudaMemcpyAsync(tot, total, sizeof tot, cudaMemcpyDeviceToHost, st));
        TRY(cudaMemcpyAsync(&mr, maxrow, sizeof mr, cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        m.max_row = mr;
        m.n_pcells = N > 0 ? tot[0] : 0;
        m.n_bcells = N > 0 ? tot[1] : 0;
        if (m.n_pcells > 0) {
            TRY(cudaMalloc(&m.pcells, sizeof(int32_t) * m.n_pcells));
            k_compact<<<nblk(N), 256, 0, st>>>(N, isp, off, m.pcells);
        }
        if (m.n_bcells > 0) {
            TRY(cudaMalloc(&m.bcells, sizeof(int32_t) * m.n_bcells));
            k_compact<<<nblk(N), 256, 0, st>>>(N, isb, offb, m.bcells);
        }
        TRY(cudaGetLastError());
        TRY(cudaStreamSynchronize(st));
    }
done:
    cudaFreeAsync(off, st);
    cudaFreeAsync(offb, st);
    cudaFreeAsync(scratch, st);
    cudaFreeAsync(total, st);
    cudaFreeAsync(key, st);
    cudaFreeAsync(bidx, st);
    cudaFreeAsync(fill, st);
    cudaFreeAsync(isp, st);
    cudaFreeAsync(isb, st);
    cudaFreeAsync(maxrow, st);
#undef TRY
    return e;
}

// ---------------------------------------------------------------------------------------------
// K1: classify every face side for every direction and count upwind dependencies n(c, Omega)
// (Alg. 2, first loop). Thread per (cell, direction); a warp reads one cell's row once.
// Tasks with no upwind cell form level 0.
// ---------------------------------------------------------------------------------------------
namespace {

// info[c][d] = {n(c, Omega): upwind interior cells,
//               P_c: FP32 projected outflow area (sign bit set when the row has more than 32 sides),
//               bit k: side k (< 32) is an inflow side (any kind),
//               bit k: side k (< 32) is an outflow side to an interior cell}
__global__ void k_classify(int64_t N, int nd, const uint32_t* rowptr, const int4* side, const d4* side64,
                           const float4* side_lo, const float4* om32, const float4* om32lo, const double* om64,
                           int4* info, int32_t* level, uint32_t* raw, int32_t* lvl_cnt, int cshift, uint32_t* dlist,
                           int32_t* n0) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool active = t < N * (int64_t)nd;
    int cnt = 0;
    uint32_t entry = 0;
    if (active) {
        int64_t c = t / nd;
        int dl = (int)(t - c * nd);
        const float4 om = om32[dl], oml = om32lo[dl];
        const double* o64 = om64 + 3 * dl;
        const uint32_t r0 = rowptr[c], r1 = rowptr[c + 1];
        float P = 0.f;
        uint32_t inm = 0u, outm = 0u;
        for (uint32_t s = r0; s < r1; ++s) {
            int4 r = side[s];
            float ax = __int_as_float(r.y), ay = __int_as_float(r.z), az = __int_as_float(r.w);
            const int sgn = classify_side(dot32(ax, ay, az, om), ax, ay, az, side64, s, o64);
            if (sgn == 0) continue;
            const uint32_t k = s - r0;
            const bool interior = r.x >= 0 && !(r.x & NBR_PERIODIC);
            if (sgn > 0) {
                P += side_weight(r, side_lo[s], om, oml);
                if (k < 32 && interior) outm |= 1u << k;
            } else {
                if (k < 32) inm |= 1u << k;
                if (interior) ++cnt;
            }
        }
        int pbits = __float_as_int(P) | ((r1 - r0 > 32u) ? (int)0x80000000 : 0);
        info[t] = make_int4(cnt, pbits, (int)inm, (int)outm);
        level[(size_t)dl * N + c] = -cnt;  // 0: level 0; the levelisation counts up to 0, then stores the level
        entry = ((uint32_t)dl << cshift) | (uint32_t)c;
    }
    bool push = active && cnt == 0;
    if (dlist) {
        // per-direction level-0 lists for the direction-parallel levelisation
        if (push) {
            const uint32_t dl = entry >> cshift;
            dlist[(size_t)dl * N + atomicAdd(&n0[dl], 1)] = entry & ~(~0u << cshift);
        }
        return;
    }
    unsigned m = __ballot_sync(0xffffffffu, push);
    if (m) {
        int lane = threadIdx.x & 31;
        int leader = __ffs(m) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&lvl_cnt[0], __popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (push) raw[base + __popc(m & ((1u << lane) - 1))] = entry;
    }
}

// ---------------------------------------------------------------------------------------------
// Direction-conserving transport (scheme (b) of Sec. 2.6), per task (c, Omega): the cell hands its
// outflow P_c I_c in equal parts to the n outflow sides whose outward normal is most nearly along
// Omega -- largest n.Omega in the exact FP64 rounding sequence of the classification, ties to the
// lower face index (rows are sorted by face) -- or to all its outflow sides if it has fewer. The share
// of each chosen side is P_c / n_c, P_c summed in FP64 in row order.
// ---------------------------------------------------------------------------------------------
constexpr int DC_MAX_N = 8;      // largest n of scheme (b)
constexpr int DC_MAX_ROW = 64;   // face sides per row (one 64-bit mask)

__global__ void k_dc_choose(int64_t N, int nd, int dcn, const uint32_t* rowptr, const d4* side64, const double* om64,
                            uint64_t* dc_mask, float* share32, double* share64, int* bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * (int64_t)nd) return;
    const int64_t c = t / nd;
    const int dl = (int)(t - c * nd);
    const uint32_t r0 = rowptr[c], r1 = rowptr[c + 1];
    if (r1 - r0 > (uint32_t)DC_MAX_ROW) {
        atomicOr(bad, 1);
        dc_mask[t] = 0ull;
        share32[t] = 0.f;
        share64[t] = 0.0;
        return;
    }
    const double* o = om64 + 3 * dl;
    double P = 0.0;
    double bt[DC_MAX_N];
    int bk[DC_MAX_N];
    int nb = 0;
    for (uint32_t s = r0; s < r1; ++s) {
        const d4 n = side64[s];
        const double tt = exact_t(n, o);
        if (!(tt > 0.0)) continue;
        P = __dadd_rn(P, __dmul_rn(n.w, tt));
        // kept sorted by (n.Omega descending, row position ascending): a later side displaces a kept one
        // only with a strictly larger n.Omega
        if (nb < dcn || tt > bt[dcn - 1]) {
            int i = nb < dcn ? nb++ : dcn - 1;
            while (i > 0 && tt > bt[i - 1]) {
                bt[i] = bt[i - 1];
                bk[i] = bk[i - 1];
                --i;
            }
            bt[i] = tt;
            bk[i] = (int)(s - r0);
        }
    }
    uint64_t m = 0ull;
    for (int i = 0; i < nb; ++i) m |= 1ull << bk[i];
    const double sh = nb > 0 ? __ddiv_rn(P, (double)nb) : 0.0;
    dc_mask[t] = m;
    share64[t] = sh;
    share32[t] = (float)sh;
}

// Effective inflow sides of each task under scheme (b) -- interior and periodic sides whose upwind cell
// chose the face (read through the twin side's position in the upwind row), and boundary inflow sides,
// which enter as in scheme (a) -- and the upwind count over the chosen interior faces, which seeds the
// levelisation (level = -count, level-0 lists per direction).
__global__ void k_dc_count(int64_t N, int nd, const uint32_t* rowptr, const int4* side, const d4* side64,
                           const float4* om32, const double* om64, const uint32_t* twin, const uint64_t* dc_mask,
                           uint64_t* dc_inm, int32_t* level, uint32_t* dlist, int32_t* n0) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * (int64_t)nd) return;
    const int64_t c = t / nd;
    const int dl = (int)(t - c * nd);
    const uint32_t r0 = rowptr[c], r1 = min(rowptr[c + 1], r0 + (uint32_t)DC_MAX_ROW);
    const float4 om = om32[dl];
    const double* o64 = om64 + 3 * dl;
    uint64_t inm = 0ull;
    int cnt = 0;
    for (uint32_t s = r0; s < r1; ++s) {
        const int4 r = side[s];
        const float ax = __int_as_float(r.y), ay = __int_as_float(r.z), az = __int_as_float(r.w);
        if (classify_side(dot32(ax, ay, az, om), ax, ay, az, side64, s, o64) >= 0) continue;
        const uint64_t bit = 1ull << (s - r0);
        if (r.x < 0) {
            inm |= bit;
            continue;
        }
        const uint32_t u = (uint32_t)(r.x & NBR_MASK);
        if ((dc_mask[(int64_t)u * nd + dl] >> twin[s]) & 1ull) {
            inm |= bit;
            if (!(r.x & NBR_PERIODIC)) ++cnt;
        }
    }
    dc_inm[t] = inm;
    level[(size_t)dl * N + c] = -cnt;
    if (cnt == 0) dlist[(size_t)dl * N + atomicAdd(&n0[dl], 1)] = (uint32_t)c;
}

// ---------------------------------------------------------------------------------------------
// K2: persistent level-synchronous Kahn over all directions. Level L occupies
// raw[pad_off[L] .. pad_off[L] + lvl_cnt[L]), padded to a multiple of 32 with TASK_PAD so
// that 32-task chunks never span two levels.
// ---------------------------------------------------------------------------------------------
constexpr int LQ_CAP = 4096;
constexpr int KL = 4;  // lanes per task in the levelisation
constexpr int KU = 8;  // face sides per lane per pass

struct LeveliseArgs {
    int64_t N;
    int nd;
    int cshift;
    uint32_t cmask;
    const uint32_t* rowptr;
    const int4* side;
    const d4* side64;
    const float4* om32;
    const double* om64;
    int4* info;
    int32_t* level;
    uint32_t* raw;
    int32_t* lvl_cnt;
    uint32_t* pad_off;
    int64_t* lev_chunk;
    int32_t* n_levels_out;
    GridBar* bar;
    int* err;
    long long budget;
};

__device__ __forceinline__ uint32_t round32(uint32_t x) { return (x + 31u) & ~31u; }

__global__ void __launch_bounds__(256) k_levelise(LeveliseArgs a) {
    __shared__ uint32_t s_q[LQ_CAP];
    __shared__ int s_n;
    __shared__ int s_base;
    const unsigned nblocks = gridDim.x;
    uint32_t base = 0;
    int n = ld_volatile_i32(&a.lvl_cnt[0]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.pad_off[0] = 0;
        a.lev_chunk[0] = 0;
    }
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    int L = 0;
    while (n > 0) {
        const uint32_t next_base = base + round32((uint32_t)n);
        if (blockIdx.x == 0)
            for (uint32_t i = base + n + threadIdx.x; i < next_base; i += blockDim.x) a.raw[i] = TASK_PAD;
        // KL lanes per task: lane j of a group owns the sides r0 + j + k*KL, loaded together; the
        // counter decrements of a pass are issued together too
        const int64_t tpb = blockDim.x / KL;  // tasks per block per round
        const int64_t tpg = (int64_t)nblocks * tpb;
        const int gl = threadIdx.x % KL;
        for (int64_t i0 = (int64_t)blockIdx.x * tpb; i0 < n; i0 += tpg) {
            const int64_t i = i0 + threadIdx.x / KL;
            if (i < n) {
                const uint32_t e = a.raw[base + i];
                const uint32_t c = e & a.cmask;
                const uint32_t dl = e >> a.cshift;
                const float4 om = a.om32[dl];
                const double* o64 = a.om64 + 3 * dl;
                const uint32_t r0 = a.rowptr[c], r1 = a.rowptr[c + 1];
                // downwind interior sides among the first 32 come from the classification mask;
                // sides past 32 (rare) are classified here
                const uint32_t outm = (uint32_t)a.info[(int64_t)c * a.nd + dl].w;
                for (uint32_t b = r0; b < r1; b += KL * KU) {
                    int4 r[KU];
#pragma unroll
                    for (int k = 0; k < KU; ++k) {
                        const uint32_t s = b + gl + k * KL;
                        const uint32_t idx = s - r0;
                        const bool need = s < r1 && (idx >= 32u || ((outm >> idx) & 1u));
                        r[k] = need ? a.side[s] : make_int4(-1, 0, 0, 0);
                    }
                    int old[KU];
#pragma unroll
                    for (int k = 0; k < KU; ++k) {
                        old[k] = 0;
                        const uint32_t s = b + gl + k * KL;
                        if (r[k].x < 0 || (r[k].x & NBR_PERIODIC)) continue;
                        if (s - r0 >= 32u) {
                            const float ax = __int_as_float(r[k].y), ay = __int_as_float(r[k].z),
                                        az = __int_as_float(r[k].w);
                            if (classify_side(dot32(ax, ay, az, om), ax, ay, az, a.side64, s, o64) <= 0) continue;
                        }
                        old[k] = atomicSub(&a.info[(int64_t)r[k].x * a.nd + dl].x, 1);
                    }
#pragma unroll
                    for (int k = 0; k < KU; ++k) {
                        if (old[k] != 1) continue;
                        a.level[(size_t)dl * a.N + (uint32_t)r[k].x] = L + 1;
                        const uint32_t ne = (dl << a.cshift) | (uint32_t)r[k].x;
                        const int p = atomicAdd(&s_n, 1);
                        if (p < LQ_CAP) s_q[p] = ne;
                        else a.raw[next_base + atomicAdd(&a.lvl_cnt[L + 1], 1)] = ne;
                    }
                }
            }
            __syncthreads();
            int cnt = s_n < LQ_CAP ? s_n : LQ_CAP;
            if (cnt > LQ_CAP / 2 || i0 + tpg >= n) {
                if (threadIdx.x == 0) s_base = cnt ? atomicAdd(&a.lvl_cnt[L + 1], cnt) : 0;
                __syncthreads();
                for (int j = threadIdx.x; j < cnt; j += blockDim.x) a.raw[next_base + s_base + j] = s_q[j];
                __syncthreads();
                if (threadIdx.x == 0) s_n = 0;
                __syncthreads();
            }
        }
        if (!grid_sync(a.bar, nblocks, a.budget, a.err)) return;
        n = ld_relaxed_i32(&a.lvl_cnt[L + 1]);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.pad_off[L + 1] = next_base;
            a.lev_chunk[L + 1] = next_base / 32;
        }
        base = next_base;
        ++L;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.n_levels_out = L;
}

// Group each level's tasks by direction (one block per level); records per-(level, direction)
// segment starts. Order inside a segment does not matter: tasks of one level are independent.
__global__ void k_sort_levels(const uint32_t* raw, uint32_t* task, const uint32_t* pad_off, const int32_t* lvl_cnt,
                              int nd, int cshift, uint32_t* seg_off, uint32_t cmask, const uint32_t* rowptr,
                              const int4* info, int4* trec) {
    extern __shared__ int s_hist[];  // 2 * nd
    const int L = blockIdx.x;
    const uint32_t b0 = pad_off[L];
    const int n = lvl_cnt[L];
    int* fill = s_hist + nd;
    for (int i = threadIdx.x; i < nd; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&s_hist[raw[b0 + i] >> cshift], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int d = 0; d < nd; ++d) {
            int h = s_hist[d];
            fill[d] = run;
            seg_off[(int64_t)L * (nd + 1) + d] = b0 + run;
            run += h;
        }
        seg_off[(int64_t)L * (nd + 1) + nd] = b0 + run;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        uint32_t e = raw[b0 + i];
        const uint32_t dl = e >> cshift, c = e & cmask;
        int p = atomicAdd(&fill[dl], 1);
        task[b0 + p] = e;
        const int4 inf = info[(int64_t)c * nd + dl];
        trec[b0 + p] = make_int4((int)e, (int)rowptr[c], inf.y, inf.z);
    }
    uint32_t end = round32((uint32_t)n);
    for (uint32_t i = n + threadIdx.x; i < end; i += blockDim.x) {
        task[b0 + i] = TASK_PAD;
        trec[b0 + i] = make_int4((int)TASK_PAD, 0, 0, 0);
    }
}

// ---------------------------------------------------------------------------------------------
// K2, direction-parallel form: the dependency graphs of different directions share nothing, so
// one block levelises one direction at a time (Alg. 2 applied level by level): the cells of level L
// release their downwind cells, a counter reaching zero puts the cell on level L+1. Levels are
// separated by __syncthreads only -- no grid barrier and no device-wide queue -- and each level's
// list is kept in shared memory (spilling to the direction's list in global memory when wide).
// ---------------------------------------------------------------------------------------------
constexpr int LD_THREADS = 1024;
constexpr int LD_KL = 4;     // lanes per task: one pass covers 32 face sides, so nearly every row takes one
constexpr int LD_KU = 8;     // face sides per lane per pass
constexpr int LD_Q = 8192;   // level-list entries {cell, row start, row end} held in shared memory (2 x 96 KB)
constexpr size_t LD_SMEM = sizeof(uint32_t) * 3 * 2 * LD_Q;

struct DirLevArgs {
    int64_t N;
    int nd;
    int cap;                 // levels the per-direction tables hold
    const uint32_t* rowptr;
    const int4* side;
    const d4* side64;
    const int2* nbr_rows;    // [S] row bounds of each side's interior neighbour
    const float4* om32;
    const double* om64;
    const uint64_t* dc_mask; // scheme (b): [N][nd] chosen outflow sides (release only those), or null
    int32_t* level;          // [nd][N]: minus the unsolved upwind cells, then the level
    uint32_t* dlist;         // [nd][N] cells of each direction in level order; level 0 from the classification
    const int32_t* n0;       // [nd] level-0 sizes
    int32_t* dcnt;           // [nd][cap] cells on each level
    int32_t* dbase;          // [nd][cap] start of each level in dlist
    int32_t* depth;          // [nd]
    int32_t* overflow;       // set when a direction has more than cap levels
};

// Per level and task: the side records of the cell's row (classified in registers: sign of n.Omega
// as in the classification) and, for each downwind interior neighbour, one atomic on its counter
// together with a load of that neighbour's row bounds, so a cell released here enters the next
// level's list with its row already known (and its row prefetched into L2 by the bulk-copy engine, so
// the next level's record loads are L2 hits): two dependent memory round trips per level.
__global__ void __launch_bounds__(LD_THREADS, 1) k_levelise_dir(DirLevArgs a) {
    extern __shared__ uint32_t s_lists[];  // [2][LD_Q][3]
    __shared__ int s_next;
    const int gl = threadIdx.x % LD_KL;
    constexpr int TPR = LD_THREADS / LD_KL;  // tasks per round
    for (int d = blockIdx.x; d < a.nd; d += gridDim.x) {
        uint32_t* out = a.dlist + (size_t)d * a.N;
        int32_t* lv = a.level + (size_t)d * a.N;
        int32_t* cnt = a.dcnt + (size_t)d * a.cap;
        int32_t* bas = a.dbase + (size_t)d * a.cap;
        const float4 om = a.om32[d];
        const double* o64 = a.om64 + 3 * d;
        int n = a.n0[d];
        for (int i = threadIdx.x; i < n && i < LD_Q; i += LD_THREADS) {
            const uint32_t c = out[i];
            s_lists[3 * i] = c;
            s_lists[3 * i + 1] = a.rowptr[c];
            s_lists[3 * i + 2] = a.rowptr[c + 1];
        }
        uint32_t base = 0;
        int L = 0, cur = 0;
        while (n > 0) {
            if (L >= a.cap) {
                if (threadIdx.x == 0) atomicExch(a.overflow, 1);
                break;
            }
            if (threadIdx.x == 0) {
                cnt[L] = n;
                bas[L] = (int32_t)base;
                s_next = 0;
            }
            __syncthreads();
            const uint32_t nbase = base + (uint32_t)n;
            const uint32_t* q = s_lists + cur * 3 * LD_Q;
            uint32_t* qn = s_lists + (cur ^ 1) * 3 * LD_Q;
            for (int i0 = 0; i0 < n; i0 += TPR) {
                const int i = i0 + threadIdx.x / LD_KL;
                if (i >= n) continue;
                uint32_t r0, r1, cc;
                if (i < LD_Q) {
                    cc = q[3 * i];
                    r0 = q[3 * i + 1];
                    r1 = q[3 * i + 2];
                } else {  // a level wider than the shared list: cells from the global list
                    cc = out[base + i];
                    r0 = a.rowptr[cc];
                    r1 = a.rowptr[cc + 1];
                }
                const uint64_t chosen = a.dc_mask ? a.dc_mask[(int64_t)cc * a.nd + d] : 0ull;
                for (uint32_t b = r0; b < r1; b += LD_KL * LD_KU) {
                    int4 r[LD_KU];
#pragma unroll
                    for (int k = 0; k < LD_KU; ++k) {
                        const uint32_t s = b + gl + k * LD_KL;
                        r[k] = s < r1 ? a.side[s] : make_int4(-1, 0, 0, 0);
                    }
                    int old[LD_KU];
                    int2 nr[LD_KU];
#pragma unroll
                    for (int k = 0; k < LD_KU; ++k) {
                        old[k] = 0;
                        nr[k] = make_int2(0, 0);
                        if (r[k].x < 0 || (r[k].x & NBR_PERIODIC)) continue;
                        const uint32_t s = b + gl + k * LD_KL;
                        const float ax = __int_as_float(r[k].y), ay = __int_as_float(r[k].z),
                                    az = __int_as_float(r[k].w);
                        if (a.dc_mask) {  // scheme (b): the chosen sides only
                            if (!((chosen >> (s - r0)) & 1ull)) continue;
                        } else if (classify_side(dot32(ax, ay, az, om), ax, ay, az, a.side64, s, o64) <= 0) {
                            continue;
                        }
                        old[k] = atomicAdd(&lv[r[k].x], 1);
                        nr[k] = a.nbr_rows[s];
                    }
#pragma unroll
                    for (int k = 0; k < LD_KU; ++k) {
                        if (old[k] != -1) continue;  // this side solved the neighbour's last upwind cell
                        const uint32_t x = (uint32_t)r[k].x;
                        lv[x] = L + 1;
                        const int p = atomicAdd(&s_next, 1);
                        if (nbase + (uint32_t)p < (uint32_t)a.N) out[nbase + p] = x;
                        if (p < LD_Q) {
                            qn[3 * p] = x;
                            qn[3 * p + 1] = (uint32_t)nr[k].x;
                            qn[3 * p + 2] = (uint32_t)nr[k].y;
                        }
                        // its side records are read on the next level: start pulling them into L2 now
                        if (nr[k].y > nr[k].x)
                            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.side + nr[k].x),
                                         "r"((uint32_t)(nr[k].y - nr[k].x) * 16u));
                    }
                }
            }
            __syncthreads();
            n = s_next;
            base = nbase;
            cur ^= 1;
            ++L;
            __syncthreads();  // everyone has read s_next before it is reset
        }
        if (threadIdx.x == 0) a.depth[d] = L;
        __syncthreads();
    }
}

// Each direction's level-ordered list rewritten with the cells of every level in cell order (the mesh's
// Hilbert order, so the tasks of a level that share upwind cells lie close together in the sweep):
// threads over (direction, cell) in cell order take the next position of their level.
__global__ void k_order_levels(int64_t N, int nd, int cap, const int32_t* level, const int32_t* dbase,
                               int32_t* fill, uint32_t* dlist) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = N * (int64_t)nd;
    const int64_t d = t < tot ? t / N : -1, c = t - d * N;
    int L = t < tot ? level[t] : -1;
    if (L >= cap) L = -1;  // negative: never levelised (a cycle) or past the tables
    // lanes of one direction and level take consecutive positions with one atomic, in lane (cell) order
    const int64_t key = L < 0 ? -1 : d * cap + L;
    const unsigned same = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31, lead = __ffs(same) - 1;
    int p = 0;
    if (lane == lead && key >= 0) p = atomicAdd(&fill[key], __popc(same));
    p = __shfl_sync(0xffffffffu, p, lead) + __popc(same & ((1u << lane) - 1u));
    if (key >= 0) dlist[d * N + dbase[key] + p] = (uint32_t)c;
}

// Cells on each level over all directions (lvl_cnt[L]) for L < n_levels.
__global__ void k_level_totals(const int32_t* dcnt, const int32_t* depth, int nd, int cap, int n_levels,
                               int32_t* lvl_cnt) {
    const int L = blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= n_levels) return;
    int s = 0;
    for (int d = 0; d < nd; ++d)
        if (L < depth[d]) s += dcnt[(size_t)d * cap + L];
    lvl_cnt[L] = s;
}

// Start of every level in the padded task list (each level padded to 32 tasks) and its chunk
// index, by one block: pad_off[L], lev_chunk[L] for L <= n_levels.
__global__ void k_level_starts(const int32_t* lvl_cnt, int n_levels, uint32_t* pad_off, int64_t* lev_chunk) {
    __shared__ uint32_t s_sum[1024];
    const int per = (n_levels + blockDim.x - 1) / blockDim.x;
    const int i0 = threadIdx.x * per;
    uint32_t loc = 0;
    for (int i = i0; i < i0 + per && i < n_levels; ++i) loc += round32((uint32_t)lvl_cnt[i]);
    s_sum[threadIdx.x] = loc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const uint32_t v = s_sum[t];
            s_sum[t] = run;
            run += v;
        }
        pad_off[n_levels] = run;
        lev_chunk[n_levels] = run / 32;
    }
    __syncthreads();
    uint32_t run = s_sum[threadIdx.x];
    for (int i = i0; i < i0 + per && i < n_levels; ++i) {
        pad_off[i] = run;
        lev_chunk[i] = run / 32;
        run += round32((uint32_t)lvl_cnt[i]);
    }
}

// Per-(level, direction) segment starts: seg_off[L][d] = pad_off[L] + cells of directions < d.
__global__ void k_seg_starts(const int32_t* dcnt, const int32_t* depth, int nd, int cap, int n_levels,
                             const uint32_t* pad_off, uint32_t* seg_off) {
    const int L = blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= n_levels) return;
    uint32_t run = pad_off[L];
    for (int d = 0; d < nd; ++d) {
        seg_off[(int64_t)L * (nd + 1) + d] = run;
        if (L < depth[d]) run += (uint32_t)dcnt[(size_t)d * cap + L];
    }
    seg_off[(int64_t)L * (nd + 1) + nd] = run;
}

// One block per level: copy each direction's cells of that level into its segment of the task list,
// with the task records, and pad the level to 32 tasks.
__global__ void k_gather_levels(const uint32_t* dlist, const int32_t* dcnt, const int32_t* dbase,
                                const int32_t* depth, int64_t N, int nd, int cap, int cshift, const uint32_t* pad_off,
                                const int32_t* lvl_cnt, const uint32_t* seg_off, const uint32_t* rowptr,
                                const int4* info, uint32_t* task, int4* trec) {
    const int L = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int d = warp; d < nd; d += nw) {
        if (L >= depth[d]) continue;
        const int n = dcnt[(size_t)d * cap + L];
        const uint32_t* src = dlist + (size_t)d * N + dbase[(size_t)d * cap + L];
        const uint32_t dst = seg_off[(int64_t)L * (nd + 1) + d];
        for (int i = lane; i < n; i += 32) {
            const uint32_t c = src[i];
            const uint32_t e = ((uint32_t)d << cshift) | c;
            const int4 inf = info[(int64_t)c * nd + d];
            task[dst + i] = e;
            trec[dst + i] = make_int4((int)e, (int)rowptr[c], inf.y, inf.z);
        }
    }
    const uint32_t b0 = pad_off[L] + (uint32_t)lvl_cnt[L], b1 = pad_off[L + 1];
    for (uint32_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        task[i] = TASK_PAD;
        trec[i] = make_int4((int)TASK_PAD, 0, 0, 0);
    }
}

// Assembled transport operator: one 128-byte line per task, in sweep order (row t of the
// lower-triangular system L_Omega I = q of Sec. 2.3, its diagonal P_c plus kappa_t V_c completed
// from the material at sweep time):
//   int4 header  {task entry, P_c (FP32 bits), n_in | boundary-entry mask << 16, destination}
//                n_in = inflow sides (capped at 255; > OP_MAX: the line is incomplete and the task
//                takes the geometry path); destination = element index dl*N + c of the intensity
//   int2 entry[OP_MAX] {source index, FP32 weight |A_f n_f.Omega|}, inflow sides in row order:
//                interior upwind cell: index dl*N + nb into this sweep's intensities, weight >= +0;
//                periodic partner: index dl*N + partner into the previous iteration's intensities,
//                weight with its sign bit set; boundary face b: index b into the boundary inflow,
//                weight with its sign bit set and the entry's bit set in the boundary mask.
//                Unused entries are {0, 0}.
// One task's line built by one thread: rows longer than 32 sides (inflow mask plus classification of
// the sides past 32), and the reference form of the assembly.
__device__ void build_line_serial(const int4 tr, int4* line, const uint32_t* rowptr, const int4* side, const d4* side64,
                                  const float4* side_lo, const float4* om32, const float4* om32lo, const double* om64,
                                  uint32_t cmask, int cshift, uint32_t N) {
    int2* E = reinterpret_cast<int2*>(line + 1);
    const uint32_t c = (uint32_t)tr.x & cmask, dl = (uint32_t)tr.x >> cshift;
    const uint32_t slab = dl * N;
    const uint32_t r0 = (uint32_t)tr.y;
    const float4 om = om32[dl], oml = om32lo[dl];
    const double* o64 = om64 + 3 * dl;
    int nin = 0;
    uint32_t bmask = 0;
    auto put = [&](const int4& r, uint32_t s) {
        if (nin < OP_MAX) {
            const float w = side_weight(r, side_lo[s], om, oml);
            int2 v;
            if (r.x >= 0 && !(r.x & NBR_PERIODIC)) {
                v = make_int2((int)(slab + (uint32_t)r.x), __float_as_int(w));
            } else if (r.x >= 0) {
                v = make_int2((int)(slab + (uint32_t)(r.x & NBR_MASK)), __float_as_int(-w));
            } else {
                v = make_int2(-1 - r.x, __float_as_int(-w));
                bmask |= 1u << nin;
            }
            E[nin] = v;
        }
        ++nin;
    };
    for (uint32_t m = (uint32_t)tr.w; m; m &= m - 1) {
        const uint32_t s = r0 + (uint32_t)(__ffs(m) - 1);
        put(side[s], s);
    }
    if (tr.z < 0) {  // rows longer than 32 sides
        const uint32_t r1 = rowptr[c + 1];
        for (uint32_t s = r0 + 32; s < r1; ++s) {
            const int4 r = side[s];
            const float ax = __int_as_float(r.y), ay = __int_as_float(r.z), az = __int_as_float(r.w);
            if (classify_side(dot32(ax, ay, az, om), ax, ay, az, side64, s, o64) >= 0) continue;
            put(r, s);
        }
    }
    for (int j = nin; j < OP_MAX; ++j) E[j] = make_int2(0, 0);
    line[0] = make_int4(tr.x, tr.z & 0x7fffffff, (nin < 255 ? nin : 255) | (int)(bmask << 16), (int)(slab + c));
}

// 8 lanes per task: lane 0 writes the header, lane g >= 1 the entries 2g-2 and 2g-1 (the (2g-2)-th and
// (2g-1)-th inflow sides of the row in row order), so the side loads of a row run in parallel and the
// 128-byte line is one coalesced store of the group. Rows longer than 32 sides take the serial form.
__global__ void __launch_bounds__(256) k_build_op(const int4* trec, int64_t n, const uint32_t* rowptr, const int4* side,
                                                  const d4* side64, const float4* side_lo, const float4* om32,
                                                  const float4* om32lo, const double* om64, uint32_t cmask, int cshift,
                                                  uint32_t N, int4* op) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;  // task
    const int gl = threadIdx.x & 7;
    const unsigned gmask = 0xffu << (threadIdx.x & 24);  // the 8 lanes of this task
    if (i >= n) return;  // a whole group at a time
    const int4 tr = trec[i];
    int4* line = op + i * 8;
    if ((uint32_t)tr.x == TASK_PAD) {
        line[gl] = gl == 0 ? make_int4((int)TASK_PAD, 0, 0, 0) : make_int4(0, 0, 0, 0);
        return;
    }
    if (tr.z < 0) {
        if (gl == 0) build_line_serial(tr, line, rowptr, side, side64, side_lo, om32, om32lo, om64, cmask, cshift, N);
        return;
    }
    const uint32_t c = (uint32_t)tr.x & cmask, dl = (uint32_t)tr.x >> cshift;
    const uint32_t slab = dl * N;
    const uint32_t r0 = (uint32_t)tr.y;
    const uint32_t inm = (uint32_t)tr.w;
    const int nin = __popc(inm);
    int2 ent[2] = {make_int2(0, 0), make_int2(0, 0)};
    uint32_t bm = 0;
    if (gl > 0) {
        const float4 om = om32[dl], oml = om32lo[dl];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int j = 2 * gl - 2 + k;
            if (j >= nin || j >= OP_MAX) continue;
            uint32_t m = inm;
            for (int q = 0; q < j; ++q) m &= m - 1;  // the j-th inflow side
            const uint32_t s = r0 + (uint32_t)(__ffs(m) - 1);
            const int4 r = side[s];
            const float w = side_weight(r, side_lo[s], om, oml);
            if (r.x >= 0 && !(r.x & NBR_PERIODIC)) {
                ent[k] = make_int2((int)(slab + (uint32_t)r.x), __float_as_int(w));
            } else if (r.x >= 0) {
                ent[k] = make_int2((int)(slab + (uint32_t)(r.x & NBR_MASK)), __float_as_int(-w));
            } else {
                ent[k] = make_int2(-1 - r.x, __float_as_int(-w));
                bm |= 1u << j;
            }
        }
    }
    bm |= __shfl_xor_sync(gmask, bm, 1);
    bm |= __shfl_xor_sync(gmask, bm, 2);
    bm |= __shfl_xor_sync(gmask, bm, 4);
    line[gl] = gl == 0 ? make_int4(tr.x, tr.z & 0x7fffffff, nin | (int)(bm << 16), (int)(slab + c))
                       : make_int4(ent[0].x, ent[0].y, ent[1].x, ent[1].y);
}

}  // namespace

cudaError_t build_operator(const DevMesh& m, const Levels& L, const double* om64_all, const float4* om32_all,
                           const float4* om32lo_all, cudaStream_t st) {
    const int64_t n = L.h_lev_chunk.empty() ? 0 : L.h_lev_chunk.back() * 32;
    if (n > 0)
        k_build_op<<<nblk(n * 8), 256, 0, st>>>(L.trec, n, m.rowptr, m.side, m.side64, m.side_lo, om32_all + L.d0,
                                            om32lo_all + L.d0, om64_all + 3 * (int64_t)L.d0, L.cmask, L.cshift,
                                            (uint32_t)m.N, L.op);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Packed operator: the rows of L_Omega (Sec. 2.3: row t = task (c, Omega), its inflow entries in
// row order and its diagonal P_c) packed back to back into 512-byte packets, so that a warp step
// streams no empty entry slots and every lane gathers. A packet is 32 lanes x 16 bytes; lane l holds
// slots 2l and 2l+1 (int2 {source, weight}):
//   a task with n inflow entries takes ceil((n + 1) / 2) consecutive lanes: entries 0..n-1 in the
//   first slots, then (n even) one empty slot {0, 0}, then its header {task entry, P_c} in the odd
//   slot of its last lane (its "head" lane);
//   entry {dl*N + nb, +w}: interior upwind cell, this sweep's intensities; {dl*N + partner, -w}:
//   periodic partner, the previous iteration's intensities; {b | PK_BOUNDARY, -w}: boundary face b,
//   the boundary inflow; w = |A_f n_f.Omega| in FP32 (the same weight as the 128-byte line);
//   the inflow sides of a row longer than 32 sides are completed by classifying the sides past 32.
// Per packet, meta = {head mask (bit l: lane l is a head lane), 1 if a task spans more than 16 lanes}.
// Tasks are packed in sweep order, next-fit, within packing groups of up to 32 chunks (1024 tasks)
// of one level; a group's packet count is rounded up to even with an empty packet, so that two
// consecutive packets of a warp step always belong to one level (independent tasks).
// The transposed operator (rows of L_Omega^T, the adjoint sweep) has the same layout: a task's
// entries are its outflow sides to interior cells {dl*N + nb, +w} and periodic partners
// {dl*N + partner, -w} (the previous pass of the transposed periodic iteration), its header the same
// {task entry, P_c}, and the levels are streamed in reverse order (downwind cells first).
// ---------------------------------------------------------------------------------------------
namespace {

constexpr int PK_GROUP_CHUNKS = 32;

struct PackArgs {
    const int4* trec;
    const int2* grp;     // [ng] {first chunk, end chunk} of each group
    int64_t ng;
    int transposed;      // the adjoint's operator: outflow entries (interior and periodic sides)
    const uint32_t* rowptr;
    const int4* side;
    const d4* side64;
    const float4* side_lo;
    const float4* om32;
    const float4* om32lo;
    const double* om64;
    uint32_t cmask;
    int cshift;
    uint32_t N;
    int32_t* cnt;        // count pass: packets per group
    int32_t* flag;       // count pass: set when a task has more than PK_MAX_IN inflow sides
    int nd;
    const uint64_t* dc_inm;   // scheme (b): [N][nd] effective inflow sides, or null (scheme (a))
    const float* dc_share32;  // scheme (b): [N][nd] share of each chosen side
    const int64_t* off;  // write pass: first packet of each group
    int4* pk;
    uint2* meta;
};

// inflow sides of a row past its first 32 (rows longer than 32 sides; their sign as in k_classify)
__device__ int pk_inflow_past32(const PackArgs& a, const int4 tr, int stop_at, uint32_t* side_out) {
    const uint32_t e = (uint32_t)tr.x, c = e & a.cmask, dl = e >> a.cshift;
    const float4 om = a.om32[dl];
    const double* o64 = a.om64 + 3 * dl;
    const uint32_t r0 = (uint32_t)tr.y, r1 = a.rowptr[c + 1];
    int k = 0;
    for (uint32_t s = r0 + 32; s < r1; ++s) {
        const int4 r = a.side[s];
        const float ax = __int_as_float(r.y), ay = __int_as_float(r.z), az = __int_as_float(r.w);
        if (classify_side(dot32(ax, ay, az, om), ax, ay, az, a.side64, s, o64) >= 0) continue;
        if (k == stop_at) {
            *side_out = s;
            return k;
        }
        ++k;
    }
    return k;
}

// outflow sides of a task's row to interior cells or periodic partners, in row order (the transposed
// operator's entries, their sign as in k_classify): their count, or the stop_at-th in *side_out
__device__ int pk_outflow(const PackArgs& a, const int4 tr, int stop_at, uint32_t* side_out) {
    const uint32_t e = (uint32_t)tr.x, c = e & a.cmask, dl = e >> a.cshift;
    const float4 om = a.om32[dl];
    const double* o64 = a.om64 + 3 * dl;
    const uint32_t r0 = (uint32_t)tr.y, r1 = a.rowptr[c + 1];
    int k = 0;
    for (uint32_t s = r0; s < r1; ++s) {
        const int4 r = a.side[s];
        if (r.x < 0) continue;  // boundary face: nothing flows back in through the transpose
        const float ax = __int_as_float(r.y), ay = __int_as_float(r.z), az = __int_as_float(r.w);
        if (classify_side(dot32(ax, ay, az, om), ax, ay, az, a.side64, s, o64) <= 0) continue;
        if (k == stop_at) {
            *side_out = s;
            return k;
        }
        ++k;
    }
    return k;
}

// scheme (b) table index of a task
__device__ __forceinline__ int64_t pk_dc_index(const PackArgs& a, uint32_t e) {
    return (int64_t)(e & a.cmask) * a.nd + (e >> a.cshift);
}

// inflow entries of a task
__device__ __forceinline__ int pk_task_inflow(const PackArgs& a, const int4 tr) {
    if (a.transposed) {
        uint32_t dummy;
        return pk_outflow(a, tr, -1, &dummy);
    }
    if (a.dc_inm) return __popcll(a.dc_inm[pk_dc_index(a, (uint32_t)tr.x)]);
    int n = __popc((uint32_t)tr.w);
    if (tr.z < 0) {
        uint32_t dummy;
        n += pk_inflow_past32(a, tr, -1, &dummy);
    }
    return n;
}

__device__ __forceinline__ int nth_set_bit(uint32_t m, int j) {
    for (int q = 0; q < j; ++q) m &= m - 1;
    return __ffs(m) - 1;
}

// entry j of a task: its j-th inflow side in row order (scheme (b): of its effective inflow sides, the
// interior and periodic ones weighted by the upwind cell's share)
__device__ int2 pk_entry(const PackArgs& a, const int4 tr, int j, uint32_t slab, const float4& om, const float4& oml) {
    uint32_t s = 0;
    if (a.transposed) {
        pk_outflow(a, tr, j, &s);
    } else if (a.dc_inm) {
        uint64_t m = a.dc_inm[pk_dc_index(a, (uint32_t)tr.x)];
        for (int q = 0; q < j; ++q) m &= m - 1;
        s = (uint32_t)tr.y + (uint32_t)(__ffsll((long long)m) - 1);
    } else {
        const uint32_t inm = (uint32_t)tr.w;
        const int nm = __popc(inm);
        if (j < nm) s = (uint32_t)tr.y + (uint32_t)nth_set_bit(inm, j);
        else pk_inflow_past32(a, tr, j - nm, &s);
    }
    const int4 r = a.side[s];
    float w = side_weight(r, a.side_lo[s], om, oml);
    if (a.dc_inm && r.x >= 0) w = a.dc_share32[(int64_t)(r.x & NBR_MASK) * a.nd + ((uint32_t)tr.x >> a.cshift)];
    if (r.x >= 0 && !(r.x & NBR_PERIODIC)) return make_int2((int)(slab + (uint32_t)r.x), __float_as_int(w));
    if (r.x >= 0) return make_int2((int)(slab + (uint32_t)(r.x & NBR_MASK)), __float_as_int(-w));
    return make_int2((int)((uint32_t)(-1 - r.x) | PK_BOUNDARY), __float_as_int(-w));
}

// One warp per packing group. The tasks of the group are read 32 at a time (lane i: task i); a
// warp prefix sum of their lane counts places them next-fit: every round closes at most one packet.
// The count pass only counts packets; the write pass repeats the same placement, hands each packet
// lane its task by shuffles, and writes the packet (16 bytes per lane, one coalesced store).
template <bool WRITE>
__global__ void __launch_bounds__(256) k_pack(PackArgs a) {
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= a.ng) return;  // whole warps
    const int lane = threadIdx.x & 31;
    const int2 gr = a.grp[g];
    const int64_t t_begin = (int64_t)gr.x * 32, t_end = (int64_t)gr.y * 32;
    int64_t pkt = WRITE ? a.off[g] : 0;
    int64_t npk = 0;
    int fill = 0;  // lanes taken in the open packet
    // the task of this lane of the open packet: record, rank of this lane in the task, its entries
    int4 my_tr = make_int4((int)TASK_PAD, 0, 0, 0);
    int my_j = 0, my_n = 0;
    auto flush = [&]() {
        if (WRITE) {
            const bool valid = (uint32_t)my_tr.x != TASK_PAD;
            const int lanes = (my_n + 2) >> 1;
            const bool head = valid && my_j == lanes - 1;
            int4 out = make_int4(0, 0, 0, 0);
            if (valid) {
                const uint32_t dl = (uint32_t)my_tr.x >> a.cshift;
                const uint32_t slab = dl * a.N;
                const float4 om = a.om32[dl], oml = a.om32lo[dl];
                const int j0 = 2 * my_j;
                const int2 s0 = j0 < my_n ? pk_entry(a, my_tr, j0, slab, om, oml) : make_int2(0, 0);
                const int2 s1 = head ? make_int2(my_tr.x, my_tr.z & 0x7fffffff)
                                     : (j0 + 1 < my_n ? pk_entry(a, my_tr, j0 + 1, slab, om, oml) : make_int2(0, 0));
                out = make_int4(s0.x, s0.y, s1.x, s1.y);
            }
            const unsigned hm = __ballot_sync(0xffffffffu, head);
            const unsigned lng = __ballot_sync(0xffffffffu, head && lanes > 16);
            a.pk[pkt * 32 + lane] = out;
            if (lane == 0) a.meta[pkt] = make_uint2(hm, lng ? 1u : 0u);
            ++pkt;
            my_tr = make_int4((int)TASK_PAD, 0, 0, 0);
        }
        ++npk;
        fill = 0;
    };
    for (int64_t t0 = t_begin; t0 < t_end; t0 += 32) {
        const int4 tr = a.trec[t0 + lane];
        const bool valid = (uint32_t)tr.x != TASK_PAD;
        int n = valid ? pk_task_inflow(a, tr) : 0;
        if (n > PK_MAX_IN) {
            if (!WRITE) atomicOr(a.flag, 1);
            n = PK_MAX_IN;  // the plan is discarded
        }
        const int sz = valid ? (n + 2) >> 1 : 0;
        int incl = sz;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        const int excl = incl - sz;
        int base = 0;  // lanes of this batch's tasks placed so far
        unsigned todo = __ballot_sync(0xffffffffu, sz > 0);
        while (todo) {
            const bool mine = (todo >> lane) & 1u;
            const unsigned fit = __ballot_sync(0xffffffffu, mine && incl - base <= 32 - fill);
            if (fit == 0) {  // the next task does not fit: close the packet
                flush();
                continue;
            }
            const int lo = __ffs(fit) - 1, hi = 31 - __clz(fit);
            const int used = __shfl_sync(0xffffffffu, incl, hi) - base;
            if (WRITE) {
                const int start = fill + excl - base;  // first packet lane of a fitting task
                const unsigned smask = __reduce_or_sync(0xffffffffu, ((fit >> lane) & 1u) ? (1u << start) : 0u);
                const bool take = lane >= fill && lane < fill + used;
                const int k = __popc(smask & ((2u << lane) - 1u)) - 1;  // rank of this lane's task among the fitting
                const int src = take ? lo + k : lane;
                const int4 r = make_int4(__shfl_sync(0xffffffffu, tr.x, src), __shfl_sync(0xffffffffu, tr.y, src),
                                         __shfl_sync(0xffffffffu, tr.z, src), __shfl_sync(0xffffffffu, tr.w, src));
                const int s_start = __shfl_sync(0xffffffffu, start, src);
                const int s_n = __shfl_sync(0xffffffffu, n, src);
                if (take) {
                    my_tr = r;
                    my_j = lane - s_start;
                    my_n = s_n;
                }
            }
            fill += used;
            base += used;
            todo &= ~fit;
            if (fill == 32) flush();
        }
    }
    if (fill > 0) flush();
    if (npk & 1) flush();  // an empty packet: every group holds an even number
    if (!WRITE && lane == 0) a.cnt[g] = (int32_t)npk;
}

__global__ void k_lev_pk(const int32_t* lev_grp, const int64_t* off, int n, int64_t* lev_pk) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) lev_pk[i] = off[lev_grp[i]];
}

PackArgs pack_args(const DevMesh& m, const Levels& L, const PackedOp& P, bool transposed, const double* om64_all,
                   const float4* om32_all, const float4* om32lo_all) {
    PackArgs a;
    a.trec = L.trec;
    a.grp = P.grp;
    a.ng = P.ng;
    a.transposed = transposed ? 1 : 0;
    a.rowptr = m.rowptr;
    a.side = m.side;
    a.side64 = m.side64;
    a.side_lo = m.side_lo;
    a.om32 = om32_all + L.d0;
    a.om32lo = om32lo_all + L.d0;
    a.om64 = om64_all + 3 * (int64_t)L.d0;
    a.cmask = L.cmask;
    a.cshift = L.cshift;
    a.N = (uint32_t)m.N;
    a.cnt = P.cnt;
    a.flag = P.flag;
    a.nd = L.nd;
    a.dc_inm = L.transport > 0 && !transposed ? L.dc_inm : nullptr;
    a.dc_share32 = L.transport > 0 && !transposed ? L.dc_share32 : nullptr;
    a.off = P.off;
    a.pk = P.pk;
    a.meta = P.meta;
    return a;
}

}  // namespace

cudaError_t pack_plan(const DevMesh& m, const Levels& L, PackedOp& P, bool transposed, const double* om64_all,
                      const float4* om32_all, const float4* om32lo_all, cudaStream_t st, int64_t* n_pk) {
    // packing groups: runs of up to PK_GROUP_CHUNKS chunks of one level (levels are padded to chunks),
    // the levels in stream order (the transposed operator: last level first)
    const int nlev = L.n_levels;
    std::vector<int2> grp;
    std::vector<int32_t> lev_grp(nlev + 1);
    for (int i = 0; i < nlev; ++i) {
        const int l = transposed ? nlev - 1 - i : i;
        lev_grp[i] = (int32_t)grp.size();
        const int64_t c1 = L.h_lev_chunk[l + 1];
        for (int64_t c = L.h_lev_chunk[l]; c < c1; c += PK_GROUP_CHUNKS)
            grp.push_back(make_int2((int)c, (int)std::min<int64_t>(c + PK_GROUP_CHUNKS, c1)));
    }
    const int64_t ng = (int64_t)grp.size();
    lev_grp[nlev] = (int32_t)ng;
    const int64_t want = std::max<int64_t>(ng, nlev) + 2;
    cudaError_t e;
    if (want > P.grp_cap || !P.flag) {
        for (void* p : {(void*)P.grp, (void*)P.lev_grp, (void*)P.cnt, (void*)P.off, (void*)P.scan, (void*)P.lev_pk,
                        (void*)P.flag})
            if (p) cudaFree(p);
        P.grp = nullptr; P.lev_grp = nullptr; P.cnt = nullptr; P.off = nullptr; P.scan = nullptr;
        P.lev_pk = nullptr; P.flag = nullptr;
        P.grp_cap = 0;
        const int64_t cap = want + want / 4;
        if ((e = cudaMalloc(&P.grp, sizeof(int2) * cap))) return e;
        if ((e = cudaMalloc(&P.lev_grp, sizeof(int32_t) * cap))) return e;
        if ((e = cudaMalloc(&P.cnt, sizeof(int32_t) * cap))) return e;
        if ((e = cudaMalloc(&P.off, sizeof(int64_t) * cap))) return e;
        if ((e = cudaMalloc(&P.scan, sizeof(int64_t) * (cap / (SCAN_BLOCK * SCAN_ITEMS) + 2)))) return e;
        if ((e = cudaMalloc(&P.lev_pk, sizeof(int64_t) * cap))) return e;
        if ((e = cudaMalloc(&P.flag, sizeof(int32_t)))) return e;
        P.grp_cap = cap;
    }
    P.ng = ng;
    if (ng > 0 && (e = cudaMemcpyAsync(P.grp, grp.data(), sizeof(int2) * ng, cudaMemcpyHostToDevice, st))) return e;
    if ((e = cudaMemcpyAsync(P.lev_grp, lev_grp.data(), sizeof(int32_t) * lev_grp.size(), cudaMemcpyHostToDevice, st)))
        return e;
    if ((e = cudaMemsetAsync(P.flag, 0, sizeof(int32_t), st))) return e;
    if (ng > 0) {
        PackArgs a = pack_args(m, L, P, transposed, om64_all, om32_all, om32lo_all);
        k_pack<false><<<(unsigned)((ng * 32 + 255) / 256), 256, 0, st>>>(a);
        if ((e = scan_i32(P.cnt, ng, P.off, P.scan, P.off + ng, st))) return e;
    } else if ((e = cudaMemsetAsync(P.off, 0, sizeof(int64_t), st))) {
        return e;
    }
    int64_t total = 0;
    int32_t flag = 0;
    if ((e = cudaMemcpyAsync(&total, P.off + ng, sizeof total, cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaMemcpyAsync(&flag, P.flag, sizeof flag, cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaStreamSynchronize(st))) return e;
    *n_pk = flag ? -1 : total;
    return cudaSuccess;
}

cudaError_t pack_write(const DevMesh& m, const Levels& L, PackedOp& P, bool transposed, const double* om64_all,
                       const float4* om32_all, const float4* om32lo_all, cudaStream_t st) {
    PackArgs a = pack_args(m, L, P, transposed, om64_all, om32_all, om32lo_all);
    if (P.ng > 0) k_pack<true><<<(unsigned)((P.ng * 32 + 255) / 256), 256, 0, st>>>(a);
    const int nlev = L.n_levels;
    k_lev_pk<<<(nlev + 1 + 255) / 256, 256, 0, st>>>(P.lev_grp, P.off, nlev, P.lev_pk);
    return cudaGetLastError();
}

namespace {

cudaError_t classify(const DevMesh& m, Levels& L, const float4* om32, const float4* om32lo, const double* om64,
                     bool per_direction, cudaStream_t st) {
    const int64_t N = m.N;
    const int nd = L.nd;
    cudaError_t e = cudaMemsetAsync(L.lvl_cnt, 0, sizeof(int32_t) * (N + 2), st);
    if (e != cudaSuccess) return e;
    int32_t* n0 = L.dlev + (int64_t)nd * 2 * L.dlev_cap;
    if (per_direction) {
        e = cudaMemsetAsync(n0, 0, sizeof(int32_t) * (2 * nd + 1), st);  // level-0 sizes, depths, overflow
        if (e != cudaSuccess) return e;
    }
    const int64_t tot = N * (int64_t)nd;
    if (tot > 0)
        k_classify<<<nblk(tot), 256, 0, st>>>(N, nd, m.rowptr, m.side, m.side64, m.side_lo, om32, om32lo, om64,
                                               L.info, L.level, L.raw, L.lvl_cnt, L.cshift,
                                               per_direction ? L.raw : nullptr, n0);
    return cudaGetLastError();
}

cudaError_t ensure_seg(Levels& L, int nlev) {
    const int nd = L.nd;
    if ((int64_t)nlev * (nd + 1) <= L.seg_cap) return cudaSuccess;
    if (L.seg_off) cudaFree(L.seg_off);
    L.seg_off = nullptr;
    L.seg_cap = 0;
    const int64_t want = ((int64_t)nlev + nlev / 4 + 16) * (nd + 1);
    cudaError_t e = cudaMalloc(&L.seg_off, sizeof(uint32_t) * want);
    if (e != cudaSuccess) return e;
    L.seg_cap = want;
    return cudaSuccess;
}

// Direction-parallel levelisation. Sets *nlev_out, or *overflow when a direction is deeper than the
// per-direction tables (the classification counters are then spent: classify again before retrying).
cudaError_t levelise_by_direction(const DevMesh& m, Levels& L, const float4* om32, const double* om64, int dev_sms,
                                  cudaStream_t st, int* nlev_out, bool* overflow) {
    const int nd = L.nd, cap = L.dlev_cap;
    int32_t* dcnt = L.dlev;
    int32_t* dbase = dcnt + (int64_t)nd * cap;
    int32_t* n0 = dbase + (int64_t)nd * cap;
    int32_t* depth = n0 + nd;
    int32_t* ovf = depth + nd;
    DirLevArgs a;
    a.N = m.N; a.nd = nd; a.cap = cap; a.rowptr = m.rowptr; a.side = m.side; a.side64 = m.side64;
    a.nbr_rows = m.nbr_rows; a.om32 = om32; a.om64 = om64; a.level = L.level; a.dlist = L.raw; a.n0 = n0;
    a.dcnt = dcnt; a.dbase = dbase;
    a.dc_mask = L.transport > 0 ? L.dc_mask : nullptr;
    a.depth = depth; a.overflow = ovf;
    const int blocks = nd < dev_sms ? nd : dev_sms;
    cudaFuncSetAttribute(k_levelise_dir, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LD_SMEM);
    k_levelise_dir<<<blocks, LD_THREADS, LD_SMEM, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    std::vector<int32_t> h(nd + 1);
    cudaMemcpyAsync(h.data(), depth, sizeof(int32_t) * (nd + 1), cudaMemcpyDeviceToHost, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    *overflow = h[nd] != 0;
    if (*overflow) return cudaSuccess;
    int nlev = 0;
    for (int d = 0; d < nd; ++d) nlev = std::max(nlev, h[d]);
    *nlev_out = nlev;
    if (nlev == 0) {
        cudaMemsetAsync(L.pad_off, 0, sizeof(uint32_t), st);
        return cudaMemsetAsync(L.lev_chunk, 0, sizeof(int64_t), st);
    }
    // the cells of each (direction, level) in cell order
    if (!L.lfill) {
        if ((e = cudaMalloc(&L.lfill, sizeof(int32_t) * (size_t)nd * cap))) return e;
    }
    if ((e = cudaMemsetAsync(L.lfill, 0, sizeof(int32_t) * (size_t)nd * cap, st))) return e;
    const int64_t tot = m.N * (int64_t)nd;
    if (tot > 0) k_order_levels<<<nblk(tot), 256, 0, st>>>(m.N, nd, cap, L.level, dbase, L.lfill, L.raw);
    e = ensure_seg(L, nlev);
    if (e != cudaSuccess) return e;
    k_level_totals<<<nblk(nlev), 256, 0, st>>>(dcnt, depth, nd, cap, nlev, L.lvl_cnt);
    k_level_starts<<<1, 1024, 0, st>>>(L.lvl_cnt, nlev, L.pad_off, L.lev_chunk);
    k_seg_starts<<<nblk(nlev), 256, 0, st>>>(dcnt, depth, nd, cap, nlev, L.pad_off, L.seg_off);
    k_gather_levels<<<nlev, 256, 0, st>>>(L.raw, dcnt, dbase, depth, m.N, nd, cap, L.cshift, L.pad_off, L.lvl_cnt,
                                          L.seg_off, m.rowptr, L.info, L.task, L.trec);
    return cudaGetLastError();
}

// Level-synchronous levelisation of all directions at once (one cooperative grid, a grid barrier
// per level), then the per-level grouping by direction. Sets *nlev_out, or *timed_out.
cudaError_t levelise_all(const DevMesh& m, Levels& L, const float4* om32, const double* om64, int dev_sms,
                         GridBar* bar, int* err, long long budget, int64_t* d_scratch, cudaStream_t st, int* nlev_out,
                         bool* timed_out) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_levelise, 256, 0);
    if (per_sm < 1) per_sm = 1;
    const int blocks = dev_sms * per_sm;
    LeveliseArgs a;
    a.N = m.N; a.nd = L.nd; a.cshift = L.cshift; a.cmask = L.cmask; a.rowptr = m.rowptr; a.side = m.side;
    a.side64 = m.side64; a.om32 = om32; a.om64 = om64; a.info = L.info; a.level = L.level; a.raw = L.raw;
    a.lvl_cnt = L.lvl_cnt; a.pad_off = L.pad_off; a.lev_chunk = L.lev_chunk;
    a.n_levels_out = (int32_t*)d_scratch; a.bar = bar; a.err = err; a.budget = budget;
    cudaMemsetAsync(bar, 0, sizeof(GridBar), st);
    cudaMemsetAsync(d_scratch, 0, sizeof(int64_t), st);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_levelise, a);
    if (e != cudaSuccess) return e;
    int32_t nlev = 0;
    int herr = 0;
    cudaMemcpyAsync(&nlev, d_scratch, sizeof nlev, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&herr, err, sizeof herr, cudaMemcpyDeviceToHost, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    *timed_out = herr != DEV_OK;
    *nlev_out = nlev;
    if (*timed_out || nlev == 0) return cudaSuccess;
    e = ensure_seg(L, nlev);
    if (e != cudaSuccess) return e;
    k_sort_levels<<<nlev, 256, 2 * L.nd * sizeof(int), st>>>(L.raw, L.task, L.pad_off, L.lvl_cnt, L.nd, L.cshift,
                                                              L.seg_off, L.cmask, m.rowptr, L.info, L.trec);
    return cudaGetLastError();
}

}  // namespace

cudaError_t levelise(const DevMesh& m, Levels& L, const double* om64_all, const float4* om32_all,
                     const float4* om32lo_all, int dev_sms, GridBar* bar, int* err, long long budget,
                     int64_t* d_scratch, cudaStream_t st, float* t_classify, float* t_levelise, std::string* msg) {
    cudaError_t e;
    const int64_t N = m.N;
    const int nd = L.nd;
    const float4* om32 = om32_all + L.d0;
    const float4* om32lo = om32lo_all + L.d0;
    const double* om64 = om64_all + 3 * (int64_t)L.d0;
    cudaEvent_t ev[3];
    for (auto& x : ev) cudaEventCreate(&x);
    cudaEventRecord(ev[0], st);
    const bool by_dir = L.dlev != nullptr && L.dlev_cap > 0;
    e = classify(m, L, om32, om32lo, om64, by_dir, st);
    if (e != cudaSuccess) return e;
    if (L.transport > 0) {
        // scheme (b): the chosen sides and shares, then the counts and level-0 lists of its thinner graph
        if (!by_dir) {
            *msg = "direction-conserving transport needs the direction-parallel levelisation";
            L.valid = false;
            return cudaSuccess;
        }
        int* bad = reinterpret_cast<int*>(d_scratch + 2);
        int32_t* n0 = L.dlev + (int64_t)nd * 2 * L.dlev_cap;
        if ((e = cudaMemsetAsync(bad, 0, sizeof(int), st))) return e;
        if ((e = cudaMemsetAsync(n0, 0, sizeof(int32_t) * nd, st))) return e;
        const int64_t tot = N * (int64_t)nd;
        if (tot > 0) {
            k_dc_choose<<<nblk(tot), 256, 0, st>>>(N, nd, L.transport, m.rowptr, m.side64, om64, L.dc_mask,
                                                   L.dc_share32, L.dc_share64, bad);
            k_dc_count<<<nblk(tot), 256, 0, st>>>(N, nd, m.rowptr, m.side, m.side64, om32, om64, m.twin, L.dc_mask,
                                                  L.dc_inm, L.level, L.raw, n0);
        }
        int hbad = 0;
        if ((e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st))) return e;
        if ((e = cudaStreamSynchronize(st))) return e;
        if (hbad) {
            *msg = "direction-conserving transport: a row has more than 64 face sides";
            L.valid = false;
            return cudaSuccess;
        }
    }
    cudaEventRecord(ev[1], st);
    int nlev = 0;
    bool done_by_dir = false;
    if (by_dir) {
        bool overflow = false;
        e = levelise_by_direction(m, L, om32, om64, dev_sms, st, &nlev, &overflow);
        if (e != cudaSuccess) return e;
        done_by_dir = !overflow;
        if (overflow && L.transport > 0) {
            *msg = "direction-conserving transport: a direction is deeper than 65536 levels";
            L.valid = false;
            return cudaSuccess;
        }
        if (overflow) {
            e = classify(m, L, om32, om32lo, om64, false, st);
            if (e != cudaSuccess) return e;
        }
    }
    if (!done_by_dir) {
        bool timed_out = false;
        e = levelise_all(m, L, om32, om64, dev_sms, bar, err, budget, d_scratch, st, &nlev, &timed_out);
        if (e != cudaSuccess) return e;
        if (timed_out) {
            *msg = "levelisation: device wait timed out";
            L.valid = false;
            return cudaSuccess;
        }
    }
    L.n_levels = nlev;
    std::vector<int32_t> cnt(nlev > 0 ? nlev : 1);
    if (nlev > 0) cudaMemcpyAsync(cnt.data(), L.lvl_cnt, sizeof(int32_t) * nlev, cudaMemcpyDeviceToHost, st);
    L.h_lev_chunk.assign(nlev + 1, 0);
    cudaMemcpyAsync(L.h_lev_chunk.data(), L.lev_chunk, sizeof(int64_t) * (nlev + 1), cudaMemcpyDeviceToHost, st);
    L.h_seg_off.assign((size_t)nlev * (nd + 1), 0);
    if (nlev > 0)
        cudaMemcpyAsync(L.h_seg_off.data(), L.seg_off, sizeof(uint32_t) * L.h_seg_off.size(), cudaMemcpyDeviceToHost,
                        st);
    cudaEventRecord(ev[2], st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    int64_t done = 0;
    for (int i = 0; i < nlev; ++i) done += cnt[i];
    L.n_tasks = done;
    const int64_t tot = N * (int64_t)nd;
    if (done != tot) {
        *msg = "dependency graph is cyclic: " + std::to_string(tot - done) + " tasks never became ready";
        L.valid = false;
        L.n_levels = 0;
        return cudaSuccess;
    }
    L.depth.assign(nd, 0);
    for (int lv = 0; lv < nlev; ++lv)
        for (int d = 0; d < nd; ++d) {
            uint32_t a0 = L.h_seg_off[(size_t)lv * (nd + 1) + d], a1 = L.h_seg_off[(size_t)lv * (nd + 1) + d + 1];
            if (a1 > a0) L.depth[d] = lv + 1;
        }
    float ms1 = 0, ms2 = 0;
    cudaEventElapsedTime(&ms1, ev[0], ev[1]);
    cudaEventElapsedTime(&ms2, ev[1], ev[2]);
    if (t_classify) *t_classify = ms1;
    if (t_levelise) *t_levelise = ms2;
    for (auto& x : ev) cudaEventDestroy(x);
    L.valid = true;
    return cudaSuccess;
}

}  // namespace sw
