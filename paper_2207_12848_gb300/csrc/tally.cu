// FP64 tallies and the per-iteration updates around the sweep (K4, K5, K6) and the
// adjoint's gradient accumulation. Every sum runs in a fixed order, so results are
// reproducible run to run; FP64 products and sums are separately rounded (no fused
// multiply-add), the rounding sequence of the FP64 oracle.
//
//   mean intensity  J_c = (1/4pi) sum_d w_d I_c,d                     (Sec. 3.2, photon rate up to 1/13.6 eV)
//   absorbed rate   Gamma_c = kappa_a,c V_c sum_d w_d I_c,d
//   escaped         sum_d w_d sum_{boundary outflow sides} |a_f| I_c,d
//   source update   q_c = eps_c/4pi + kappa_s,c V_c J_c                (Alg. 1, scattering as a fixed source)
//   periodic source j_c = sum_d w_d sum_{periodic inflow sides} |a_f| I_partner,d   (Sec. 2.7)
//   relative change E_c = |j^n - j^(n-1)| / (j^n + j^(n-1))             (Eq. relativeErrorPbc)
#include "adjoint.cuh"
#include "common.cuh"

namespace sw {
namespace {

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }

template <typename real>
__device__ __forceinline__ double mag(const real* p) { return fabs((double)*p); }

// deterministic block sum of two values per thread into out[blockIdx][0..1]
__device__ void block_sum2(double a, double b, double* out) {
    __shared__ double s0[256], s1[256];
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = b;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            s0[threadIdx.x] += s0[threadIdx.x + off];
            s1[threadIdx.x] += s1[threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * blockIdx.x] = s0[0];
        out[2 * blockIdx.x + 1] = s1[0];
    }
}

__global__ void k_prep_material(int64_t N, int G, const double* vol, const double* ka, const double* ks,
                                const double* em, const double* J, float2* cm32, double2* cm64) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * G) return;
    int64_t c = i / G;
    double V = vol[c];
    double kscat = ks ? ks[i] : 0.0;
    double q = em[i] / FOURPI;
    if (ks && J) q = dadd(q, dmul(dmul(kscat, V), J[i]));
    double dnm = dmul(dadd(ka[i], kscat), V);
    if (cm64) cm64[i] = make_double2(q, dnm);
    if (cm32) cm32[i] = make_float2((float)q, (float)dnm);
}

// adjoint sources split into non-negative parts: groups [0,G) carry g+, [G,2G) carry g-
__global__ void k_prep_adjoint(int64_t N, int G, const double* vol, const double* ka, const double* ks,
                               const double* dlj, const double* dlg, float2* cm32, double2* cm64) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * G) return;
    int64_t c = i / G;
    int g = (int)(i - c * G);
    double V = vol[c];
    double gd = dlg ? dmul(dmul(dlg[i], ka[i]), V) : 0.0;
    double gj = dlj ? dlj[i] / FOURPI : 0.0;
    double src = dadd(gd, gj);
    double dnm = dmul(dadd(ka[i], ks ? ks[i] : 0.0), V);
    double gp = src > 0.0 ? src : 0.0, gm = src < 0.0 ? -src : 0.0;
    int64_t o = c * (2 * G);
    if (cm64) {
        cm64[o + g] = make_double2(gp, dnm);
        cm64[o + G + g] = make_double2(gm, dnm);
    }
    if (cm32) {
        cm32[o + g] = make_float2((float)gp, (float)dnm);
        cm32[o + G + g] = make_float2((float)gm, (float)dnm);
    }
}

template <typename real>
__global__ void k_tally(const real* I, int64_t N, int G, int nd, const double* w64, double wsum, const double* vol,
                        const double* ka, const double* em, double* J, double* Gam, double* partial) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double absorbed = 0.0, emitted = 0.0;
    if (i < N * G) {
        double s = 0.0;
        const size_t NG = (size_t)N * G;
        for (int d = 0; d < nd; ++d) s = dadd(s, dmul(w64[d], mag(I + d * NG + i)));
        double j = s / FOURPI;
        int64_t c = i / G;
        double gam = dmul(dmul(dmul(ka[i], vol[c]), FOURPI), j);
        J[i] = j;
        if (Gam) Gam[i] = gam;
        absorbed = gam;
        emitted = dmul(em[i], wsum) / FOURPI;
    }
    block_sum2(absorbed, emitted, partial);
}

// Sums over the rows of a few cells (boundary or periodic cells) for every direction: one block per
// cell, its threads over directions, so the FP64 classification and the strided intensity reads of
// the D directions run in parallel; the block's partial sums are then combined in a fixed order
// (warp shuffles, then the warps in index order), so results do not depend on timing.
constexpr int ROW_THREADS = 128;

__device__ __forceinline__ double block_sum_fixed(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();  // sh may still be read from the previous call
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < ROW_THREADS / 32; ++w) t += sh[w];
    return t;
}

// Escaped (outflow through vacuum faces) and injected (boundary inflow) photon rates of one boundary
// cell, into partial[2k], partial[2k+1].
template <typename real>
__global__ void __launch_bounds__(ROW_THREADS) k_boundary_tally(const int32_t* bcells, const uint32_t* rowptr,
                                                                const int4* side, const d4* side64, const real* I,
                                                                int64_t N, int G, int nd, const double* om64,
                                                                const double* w64, const double* bc,
                                                                double* partial, DcTabs dc) {
    __shared__ double sh[ROW_THREADS / 32];
    const int64_t k = blockIdx.x;
    const int32_t c = bcells[k];
    const uint32_t r0 = rowptr[c], r1 = rowptr[c + 1];
    double esc = 0.0, inj = 0.0;
    for (int d = threadIdx.x; d < nd; d += ROW_THREADS) {
        const double w = w64[d];
        for (uint32_t s = r0; s < r1; ++s) {
            const int32_t nbr = side[s].x;
            if (nbr >= 0) continue;
            const d4 n = side64[s];
            const double t = exact_t(n, om64 + 3 * d);
            const double wa = dmul(w, dmul(n.w, fabs(t)));
            // scheme (b): the outflow leaves through a vacuum face only if the cell chose it, with its share
            double wo = wa;
            if (dc.mask && t > 0.0) {
                const int64_t i = (int64_t)c * nd + d;
                wo = ((dc.mask[i] >> (s - r0)) & 1ull) ? dmul(w, dc.share64[i]) : 0.0;
            }
            for (int g = 0; g < G; ++g) {
                if (t > 0.0) esc = dadd(esc, dmul(wo, mag(I + ((size_t)d * N + c) * G + g)));
                else if (t < 0.0 && bc) inj = dadd(inj, dmul(wa, bc[(size_t)(-1 - nbr) * G + g]));
            }
        }
    }
    esc = block_sum_fixed(esc, sh);
    inj = block_sum_fixed(inj, sh);
    if (threadIdx.x == 0) {
        partial[2 * k] = esc;
        partial[2 * k + 1] = inj;
    }
}

// Periodic iteration (Sec. 2.7): the inflow j^n of one periodic cell and group, summed over the
// directions and its periodic sides of the partner cells' intensities, and the relative change
// E = |j^n - j^(n-1)| / (j^n + j^(n-1)) (Eq. relativeErrorPbc). Writes jn1, raises *dmax to the
// cell's largest E, and puts the sum of its E over groups into partial[2k].
template <typename real>
__global__ void __launch_bounds__(ROW_THREADS) k_periodic_source(const int32_t* pcells, const uint32_t* rowptr,
                                                                 const int4* side, const d4* side64, const real* I,
                                                                 int64_t N, int G, int nd, const double* om64,
                                                                 const double* w64, double* jn1, const double* jn,
                                                                 unsigned long long* dmax, double* partial) {
    __shared__ double sh[ROW_THREADS / 32];
    const int64_t k = blockIdx.x;
    const int32_t c = pcells[k];
    const uint32_t r0 = rowptr[c], r1 = rowptr[c + 1];
    double j[8];
    for (int g = 0; g < 8; ++g) j[g] = 0.0;
    for (int d = threadIdx.x; d < nd; d += ROW_THREADS) {
        const double w = w64[d];
        for (uint32_t s = r0; s < r1; ++s) {
            const int32_t nbr = side[s].x;
            if (nbr < 0 || !(nbr & NBR_PERIODIC)) continue;
            const d4 n = side64[s];
            const double t = exact_t(n, om64 + 3 * d);
            if (!(t < 0.0)) continue;
            const double wa = dmul(w, dmul(n.w, fabs(t)));
            const size_t base = ((size_t)d * N + (uint32_t)(nbr & NBR_MASK)) * G;
            for (int g = 0; g < G; ++g) j[g] = dadd(j[g], dmul(wa, mag(I + base + g)));
        }
    }
    double esum = 0.0, emax = 0.0;
    for (int g = 0; g < G; ++g) {
        const double jt = block_sum_fixed(j[g], sh);
        if (threadIdx.x == 0) {
            const size_t i = (size_t)c * G + g;
            const double s = jt + jn[i];
            const double e = s > 0.0 ? fabs(jt - jn[i]) / s : 0.0;
            jn1[i] = jt;
            esum += e;
            if (e > emax) emax = e;
        }
    }
    if (threadIdx.x == 0) {
        if (emax > 0.0) atomicMax(dmax, (unsigned long long)__double_as_longlong(emax));
        partial[2 * k] = esum;
        partial[2 * k + 1] = 0.0;
    }
}

// Periodic-inflow weight table, fixed for a solve: for every periodic side of every periodic cell (in
// row order) and every direction, w_d A |n.Omega| in FP64 where the side is an inflow side, else 0.
// Built once per solve; each iteration then needs one FP64 multiply-add per inflow side and direction
// instead of recomputing n.Omega and the weight on this part's narrow FP64 pipe.
__global__ void k_pside_count(const int32_t* pcells, int64_t np, const uint32_t* rowptr, const int4* side,
                              int32_t* cnt) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    const int32_t c = pcells[k];
    int n = 0;
    for (uint32_t s = rowptr[c]; s < rowptr[c + 1]; ++s) {
        const int32_t x = side[s].x;
        if (x >= 0 && (x & NBR_PERIODIC)) ++n;
    }
    cnt[k] = n;
}

// exclusive scan of n counts by one block of 1024 threads; off[n] = total
__global__ void k_scan_counts(const int32_t* cnt, int64_t n, int32_t* off) {
    __shared__ int32_t s_sum[1024];
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t i0 = threadIdx.x * per;
    int32_t loc = 0;
    for (int64_t i = i0; i < i0 + per && i < n; ++i) loc += cnt[i];
    s_sum[threadIdx.x] = loc;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t run = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const int32_t v = s_sum[t];
            s_sum[t] = run;
            run += v;
        }
        off[n] = run;
    }
    __syncthreads();
    int32_t run = s_sum[threadIdx.x];
    for (int64_t i = i0; i < i0 + per && i < n; ++i) {
        off[i] = run;
        run += cnt[i];
    }
}

__global__ void __launch_bounds__(ROW_THREADS) k_pside_weights(const int32_t* pcells, const int32_t* off,
                                                               const uint32_t* rowptr, const int4* side,
                                                               const d4* side64, int nd, const double* om64,
                                                               const double* w64, double* wa, DcTabs dc) {
    const int64_t k = blockIdx.x;
    const int32_t c = pcells[k];
    const uint32_t r0 = rowptr[c], r1 = rowptr[c + 1];
    for (int d = threadIdx.x; d < nd; d += ROW_THREADS) {
        int64_t j = off[k];
        for (uint32_t s = r0; s < r1; ++s) {
            const int32_t x = side[s].x;
            if (x < 0 || !(x & NBR_PERIODIC)) continue;
            const d4 n = side64[s];
            const double t = exact_t(n, om64 + 3 * d);
            double v = t < 0.0 ? dmul(w64[d], dmul(n.w, fabs(t))) : 0.0;
            if (dc.mask && t < 0.0) {  // scheme (b): the partner's share, if the partner chose this face
                const int64_t i = (int64_t)(x & NBR_MASK) * nd + d;
                v = ((dc.mask[i] >> dc.twin[s]) & 1ull) ? dmul(w64[d], dc.share64[i]) : 0.0;
            }
            wa[j * nd + d] = v;
            ++j;
        }
    }
}

// k_periodic_source with the weights from the table (same sums in the same order)
template <typename real>
__global__ void __launch_bounds__(ROW_THREADS) k_periodic_source_tab(const int32_t* pcells, const int32_t* off,
                                                                     const uint32_t* rowptr, const int4* side,
                                                                     const double* wa, const real* I, int64_t N, int G,
                                                                     int nd, double* jn1, const double* jn,
                                                                     unsigned long long* dmax, double* partial) {
    __shared__ double sh[ROW_THREADS / 32];
    const int64_t k = blockIdx.x;
    const int32_t c = pcells[k];
    const uint32_t r0 = rowptr[c], r1 = rowptr[c + 1];
    double j[8];
    for (int g = 0; g < 8; ++g) j[g] = 0.0;
    for (int d = threadIdx.x; d < nd; d += ROW_THREADS) {
        int64_t q = off[k];
        for (uint32_t s = r0; s < r1; ++s) {
            const int32_t nbr = side[s].x;
            if (nbr < 0 || !(nbr & NBR_PERIODIC)) continue;
            const double w = wa[q * nd + d];
            ++q;
            if (w == 0.0) continue;  // not an inflow side for this direction
            const size_t base = ((size_t)d * N + (uint32_t)(nbr & NBR_MASK)) * G;
            for (int g = 0; g < G; ++g) j[g] = dadd(j[g], dmul(w, mag(I + base + g)));
        }
    }
    double esum = 0.0, emax = 0.0;
    for (int g = 0; g < G; ++g) {
        const double jt = block_sum_fixed(j[g], sh);
        if (threadIdx.x == 0) {
            const size_t i = (size_t)c * G + g;
            const double s = jt + jn[i];
            const double e = s > 0.0 ? fabs(jt - jn[i]) / s : 0.0;
            jn1[i] = jt;
            esum += e;
            if (e > emax) emax = e;
        }
    }
    if (threadIdx.x == 0) {
        if (emax > 0.0) atomicMax(dmax, (unsigned long long)__double_as_longlong(emax));
        partial[2 * k] = esum;
        partial[2 * k + 1] = 0.0;
    }
}

__global__ void k_scat_residual(int64_t NG, const double* J, double* Jold, unsigned long long* dmax) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NG) return;
    double dj = fabs(J[i] - Jold[i]);
    double e;
    if (dj == 0.0) e = 0.0;
    else if (J[i] > 0.0) e = dj / J[i];
    else e = INFINITY;
    Jold[i] = J[i];
    if (e > 0.0) atomicMax(dmax, (unsigned long long)__double_as_longlong(e));
}

// sum of n pairs in a fixed order: 1024 threads, four independent accumulators each (elements i + u T,
// u = 0..3, then every 4T), combined pairwise, then a shared-memory tree
__global__ void __launch_bounds__(1024) k_reduce_sum(const double* partial, int n, double* out) {
    __shared__ double s0[1024], s1[1024];
    const int T = blockDim.x;
    double a[4] = {0.0, 0.0, 0.0, 0.0}, b[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += 4 * T) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = i + u * T;
            if (j < n) {
                a[u] += partial[2 * j];
                b[u] += partial[2 * j + 1];
            }
        }
    }
    s0[threadIdx.x] = (a[0] + a[1]) + (a[2] + a[3]);
    s1[threadIdx.x] = (b[0] + b[1]) + (b[2] + b[3]);
    __syncthreads();
    for (int off = T / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            s0[threadIdx.x] += s0[threadIdx.x + off];
            s1[threadIdx.x] += s1[threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = s0[0];
        out[1] = s1[0];
    }
}

// lambda of group g = lambda+ (group g) - lambda- (group G+g) of the split adjoint sweep. With
// scattering (J != nullptr) also dL/dkappa_s = V sum_d lambda_d (J - I_d).
template <typename real>
__global__ void k_grad(const real* I, const real* lam, int64_t N, int G, int nd, const double* w64, const double* vol,
                       const double* dlg, const double* J, double* gk, double* ge, double* gks) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * G) return;
    int64_t c = i / G;
    int g = (int)(i - c * G);
    double V = vol[c];
    double rg = dlg ? dlg[i] : 0.0;
    double Jc = J ? J[i] : 0.0;
    double sk = gk[i], se = ge[i], ss = 0.0;
    for (int d = 0; d < nd; ++d) {
        double Icd = mag(I + ((size_t)d * N + c) * G + g);
        const real* lp = lam + ((size_t)d * N + c) * (2 * G);
        double lcd = mag(lp + g) - mag(lp + G + g);
        sk = dadd(sk, dmul(dmul(V, Icd), dmul(w64[d], rg) - lcd));
        se = dadd(se, lcd / FOURPI);
        ss = dadd(ss, dmul(dmul(V, lcd), Jc - Icd));
    }
    gk[i] = sk;
    ge[i] = se;
    if (J && gks) gks[i] = ss;
}

// Transposed iteration: mu+- = sum_d lambda+-_d (no direction weight: the reverse sweep puts w_d on
// its source), the largest change and the largest magnitude of mu = mu+ - mu- (dmax[0], dmax[1]), and
// the split sources of the next transposed sweep, g+- + kappa_s V mu+- / 4pi (ks may be null).
template <typename real>
__global__ void k_adj_mu(const real* lam, int64_t N, int G, int nd, const double* vol, const double* ka,
                         const double* ks, const double* dlj, const double* dlg, double* mu, float2* cm32,
                         double2* cm64, unsigned long long* dmax) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * G) return;
    int64_t c = i / G;
    int g = (int)(i - c * G);
    const size_t G2 = 2 * (size_t)G;
    double sp = 0.0, sm = 0.0;
    for (int d = 0; d < nd; ++d) {
        const real* lp = lam + ((size_t)d * N + c) * G2;
        sp = dadd(sp, mag(lp + g));
        sm = dadd(sm, mag(lp + G + g));
    }
    const size_t o = (size_t)c * G2;
    double change = fabs((sp - sm) - (mu[o + g] - mu[o + G + g]));
    double size = fabs(sp - sm);
    mu[o + g] = sp;
    mu[o + G + g] = sm;
    if (change > 0.0) atomicMax(dmax, (unsigned long long)__double_as_longlong(change));
    if (size > 0.0) atomicMax(dmax + 1, (unsigned long long)__double_as_longlong(size));
    double V = vol[c];
    double src = dadd(dlg ? dmul(dmul(dlg[i], ka[i]), V) : 0.0, dlj ? dlj[i] / FOURPI : 0.0);
    double gp = src > 0.0 ? src : 0.0, gm = src < 0.0 ? -src : 0.0;
    double kv = ks ? dmul(ks[i], V) : 0.0;
    double qp = dadd(gp, dmul(kv, sp) / FOURPI), qm = dadd(gm, dmul(kv, sm) / FOURPI);
    double dnm = dmul(dadd(ka[i], ks ? ks[i] : 0.0), V);
    if (cm64) {
        cm64[o + g] = make_double2(qp, dnm);
        cm64[o + G + g] = make_double2(qm, dnm);
    }
    if (cm32) {
        cm32[o + g] = make_float2((float)qp, (float)dnm);
        cm32[o + G + g] = make_float2((float)qm, (float)dnm);
    }
}

__global__ void k_fill_u32(uint32_t* p, uint32_t v, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

template <typename real>
__global__ void k_to_f64(const real* I, int64_t n, double* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = fabs((double)I[i]);
}

inline unsigned nb(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_prep_material(int64_t N, int G, const double* vol, const double* ka, const double* ks,
                                 const double* em, const double* J, float2* cm32, double2* cm64, cudaStream_t st) {
    if (N * G > 0) k_prep_material<<<nb(N * G), 256, 0, st>>>(N, G, vol, ka, ks, em, J, cm32, cm64);
    return cudaGetLastError();
}

cudaError_t launch_prep_adjoint_src(int64_t N, int G, const double* vol, const double* ka, const double* ks,
                                    const double* dl_dJ, const double* dl_dG, float2* cm32, double2* cm64,
                                    cudaStream_t st) {
    if (N * G > 0) k_prep_adjoint<<<nb(N * G), 256, 0, st>>>(N, G, vol, ka, ks, dl_dJ, dl_dG, cm32, cm64);
    return cudaGetLastError();
}

cudaError_t launch_tally(int precision, const void* I, int64_t N, int G, int nd, int d0, const double* w64,
                         double wsum, const double* vol, const double* ka, const double* em, double* J, double* Gam,
                         double* partial, int nblk_, cudaStream_t st) {
    (void)nblk_;
    unsigned b = nb(N * G);
    if (b == 0) b = 1;
    if (precision == 64)
        k_tally<double><<<b, 256, 0, st>>>((const double*)I, N, G, nd, w64 + d0, wsum, vol, ka, em, J, Gam, partial);
    else
        k_tally<float><<<b, 256, 0, st>>>((const float*)I, N, G, nd, w64 + d0, wsum, vol, ka, em, J, Gam, partial);
    return cudaGetLastError();
}

cudaError_t launch_boundary_tally(int precision, const DevMesh& m, const void* I, int G, int nd, int d0,
                                  const double* om64, const double* w64, const double* bc, double* partial, int nblk_,
                                  cudaStream_t st, const DcTabs* dc) {
    (void)nblk_;
    const DcTabs tabs = dc ? *dc : DcTabs();
    if (m.n_bcells <= 0) return cudaSuccess;
    const unsigned b = (unsigned)m.n_bcells;
    if (precision == 64)
        k_boundary_tally<double><<<b, ROW_THREADS, 0, st>>>(m.bcells, m.rowptr, m.side, m.side64, (const double*)I,
                                                            m.N, G, nd, om64 + 3 * d0, w64 + d0, bc, partial, tabs);
    else
        k_boundary_tally<float><<<b, ROW_THREADS, 0, st>>>(m.bcells, m.rowptr, m.side, m.side64, (const float*)I,
                                                           m.N, G, nd, om64 + 3 * d0, w64 + d0, bc, partial, tabs);
    return cudaGetLastError();
}

cudaError_t launch_scat_residual(int64_t NG, const double* J, double* Jold, unsigned long long* d_max,
                                 cudaStream_t st) {
    if (NG > 0) k_scat_residual<<<nb(NG), 256, 0, st>>>(NG, J, Jold, d_max);
    return cudaGetLastError();
}

cudaError_t build_periodic_table(const DevMesh& m, int nd, const double* om64, const double* w64, PeriodicTable* t,
                                 cudaStream_t st, const DcTabs* dc) {
    if (m.n_pcells <= 0) return cudaSuccess;
    const int64_t np = m.n_pcells;
    cudaError_t e;
    if (t->off_cap < (size_t)(2 * (np + 1))) {
        if (t->off) cudaFree(t->off);
        t->off = nullptr;
        t->off_cap = 0;
        if ((e = cudaMalloc(&t->off, sizeof(int32_t) * 2 * (np + 1)))) return e;
        t->off_cap = 2 * (np + 1);
    }
    int32_t* cnt = t->off + (np + 1);
    k_pside_count<<<nb(np), 256, 0, st>>>(m.pcells, np, m.rowptr, m.side, cnt);
    k_scan_counts<<<1, 1024, 0, st>>>(cnt, np, t->off);
    int32_t total = 0;
    if ((e = cudaMemcpyAsync(&total, t->off + np, sizeof total, cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaStreamSynchronize(st))) return e;
    const size_t need = (size_t)(total > 0 ? total : 1) * nd;
    if (t->wa_cap < need) {
        if (t->wa) cudaFree(t->wa);
        t->wa = nullptr;
        t->wa_cap = 0;
        if ((e = cudaMalloc(&t->wa, sizeof(double) * need))) return e;
        t->wa_cap = need;
    }
    k_pside_weights<<<(unsigned)np, ROW_THREADS, 0, st>>>(m.pcells, t->off, m.rowptr, m.side, m.side64, nd, om64, w64,
                                                          t->wa, dc ? *dc : DcTabs());
    t->ready = true;
    return cudaGetLastError();
}

cudaError_t launch_periodic_source(int precision, const DevMesh& m, const void* I, int G, int nd, const double* om64,
                                   const double* w64, double* jn1, const double* jn, unsigned long long* d_max,
                                   double* partial, int nblk_, cudaStream_t st, const PeriodicTable* tab) {
    (void)nblk_;
    if (m.n_pcells <= 0) return cudaSuccess;
    const unsigned b = (unsigned)m.n_pcells;
    if (tab && tab->ready) {
        if (precision == 64)
            k_periodic_source_tab<double><<<b, ROW_THREADS, 0, st>>>(m.pcells, tab->off, m.rowptr, m.side, tab->wa,
                                                                     (const double*)I, m.N, G, nd, jn1, jn, d_max,
                                                                     partial);
        else
            k_periodic_source_tab<float><<<b, ROW_THREADS, 0, st>>>(m.pcells, tab->off, m.rowptr, m.side, tab->wa,
                                                                    (const float*)I, m.N, G, nd, jn1, jn, d_max,
                                                                    partial);
        return cudaGetLastError();
    }
    if (precision == 64)
        k_periodic_source<double><<<b, ROW_THREADS, 0, st>>>(m.pcells, m.rowptr, m.side, m.side64, (const double*)I,
                                                             m.N, G, nd, om64, w64, jn1, jn, d_max, partial);
    else
        k_periodic_source<float><<<b, ROW_THREADS, 0, st>>>(m.pcells, m.rowptr, m.side, m.side64, (const float*)I,
                                                            m.N, G, nd, om64, w64, jn1, jn, d_max, partial);
    return cudaGetLastError();
}

cudaError_t launch_reduce_sum(const double* partial, int n, double* out, cudaStream_t st) {
    k_reduce_sum<<<1, 1024, 0, st>>>(partial, n, out);
    return cudaGetLastError();
}

cudaError_t launch_grad_accum(int precision, const void* I, const void* lam, int64_t N, int G, int nd, int d0,
                              const double* w64, const double* vol, const double* dl_dG, double* gk, double* ge,
                              cudaStream_t st) {
    return launch_grad_scat(precision, I, lam, N, G, nd, d0, w64, vol, dl_dG, nullptr, gk, ge, nullptr, st);
}

cudaError_t launch_grad_scat(int precision, const void* I, const void* lam, int64_t N, int G, int nd, int d0,
                             const double* w64, const double* vol, const double* dl_dG, const double* J, double* gk,
                             double* ge, double* gks, cudaStream_t st) {
    if (N * G <= 0) return cudaSuccess;
    if (precision == 64)
        k_grad<double><<<nb(N * G), 256, 0, st>>>((const double*)I, (const double*)lam, N, G, nd, w64 + d0, vol,
                                                  dl_dG, J, gk, ge, gks);
    else
        k_grad<float><<<nb(N * G), 256, 0, st>>>((const float*)I, (const float*)lam, N, G, nd, w64 + d0, vol, dl_dG,
                                                 J, gk, ge, gks);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_mu(int precision, const void* lam, int64_t N, int G, int nd, const double* vol,
                              const double* ka, const double* ks, const double* dl_dJ, const double* dl_dG,
                              double* mu, float2* cm32, double2* cm64, unsigned long long* d_max, cudaStream_t st) {
    if (N * G <= 0) return cudaSuccess;
    if (precision == 64)
        k_adj_mu<double><<<nb(N * G), 256, 0, st>>>((const double*)lam, N, G, nd, vol, ka, ks, dl_dJ, dl_dG, mu,
                                                    cm32, cm64, d_max);
    else
        k_adj_mu<float><<<nb(N * G), 256, 0, st>>>((const float*)lam, N, G, nd, vol, ka, ks, dl_dJ, dl_dG, mu, cm32,
                                                   cm64, d_max);
    return cudaGetLastError();
}

cudaError_t launch_fill_u32(uint32_t* p, uint32_t v, int64_t n, cudaStream_t st) {
    if (n > 0) k_fill_u32<<<nb(n), 256, 0, st>>>(p, v, n);
    return cudaGetLastError();
}

cudaError_t launch_to_f64(int precision, const void* I, int64_t n, double* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (precision == 64) k_to_f64<double><<<nb(n), 256, 0, st>>>((const double*)I, n, out);
    else k_to_f64<float><<<nb(n), 256, 0, st>>>((const float*)I, n, out);
    return cudaGetLastError();
}

}  // namespace sw

// ---------------------------------------------------------------------------------------------
// Rotation of the direction set (the rotation paragraph of Sec. 2.6): the remap coefficients
// c_ij = dS_ij / dS_i between the bins of the new directions i and the old directions j, by a
// quadrature of equal-weight points on the unit sphere, and the remap of the stored intensities
// I(Omega'_i) = sum_j c_ij I(Omega_j).
// ---------------------------------------------------------------------------------------------
namespace sw {
namespace {

// the direction (of n_dir) nearest to p: largest ((px Ox) + (py Oy)) + (pz Oz), ties to the lower index
__device__ __forceinline__ int nearest_dir(const double3 p, const double* om, int n_dir) {
    int best = 0;
    double bd = -2.0;
    for (int d = 0; d < n_dir; ++d) {
        const double t = __dadd_rn(__dadd_rn(__dmul_rn(p.x, om[3 * d]), __dmul_rn(p.y, om[3 * d + 1])),
                                   __dmul_rn(p.z, om[3 * d + 2]));
        if (t > bd) {
            bd = t;
            best = d;
        }
    }
    return best;
}

__global__ void k_remap_count(const double3* pts, int64_t n, const double* om_old, const double* om_new, int n_dir,
                              unsigned long long* cnt) {
    extern __shared__ double s_om[];  // [2][n_dir][3]
    for (int i = threadIdx.x; i < 6 * n_dir; i += blockDim.x) s_om[i] = i < 3 * n_dir ? om_new[i] : om_old[i - 3 * n_dir];
    __syncthreads();
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const double3 p = pts[m];
    const int i = nearest_dir(p, s_om, n_dir);
    const int j = nearest_dir(p, s_om + 3 * n_dir, n_dir);
    atomicAdd(&cnt[(int64_t)i * n_dir + j], 1ull);
}

// out[i][c][g] = sum over the nonzeros (j, c_ij) of row i of c_ij |in[j][c][g]|, written with the sign
// bit `par` (the parity the buffer's values carry); one thread per (cell, group) element
template <typename real>
__global__ void k_remap(const real* in, real* out, int64_t NG, int n_dir, const int32_t* rp, const int32_t* col,
                        const double* val, int par) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NG) return;
    for (int i = 0; i < n_dir; ++i) {
        double acc = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k)
            acc = __dadd_rn(acc, __dmul_rn(val[k], fabs((double)in[(int64_t)col[k] * NG + e])));
        const real v = (real)acc;
        out[(int64_t)i * NG + e] = par ? -v : v;
    }
}

}  // namespace

cudaError_t launch_remap_count(const double3* pts, int64_t n, const double* om_old, const double* om_new, int n_dir,
                               unsigned long long* cnt, cudaStream_t st) {
    if (n > 0)
        k_remap_count<<<(unsigned)((n + 255) / 256), 256, sizeof(double) * 6 * n_dir, st>>>(pts, n, om_old, om_new,
                                                                                            n_dir, cnt);
    return cudaGetLastError();
}

cudaError_t launch_remap(int precision, const void* in, void* out, int64_t NG, int n_dir, const int32_t* rp,
                         const int32_t* col, const double* val, int par, cudaStream_t st) {
    if (NG <= 0) return cudaSuccess;
    const unsigned b = (unsigned)((NG + 255) / 256);
    if (precision == 64)
        k_remap<double><<<b, 256, 0, st>>>((const double*)in, (double*)out, NG, n_dir, rp, col, val, par);
    else
        k_remap<float><<<b, 256, 0, st>>>((const float*)in, (float*)out, NG, n_dir, rp, col, val, par);
    return cudaGetLastError();
}

}  // namespace sw
