// sweep_levels_noalloc: wavefront levels of one direction with no device allocation.
//
// Some callers cannot allocate GPU memory at the point where they need the sweep order: code that
// runs under a fixed device-memory budget (an arena or pool that hands out no new blocks), or next
// to a component that already holds nearly all device memory, where a cudaMalloc would fail or
// stall the device. This entry point takes the mesh and the output in the caller's own device
// buffers and keeps its working memory (upwind counters and a small control block) in one
// file-scope device array, reserved when the library's module is loaded and held by every GPU that
// loads it until the process exits.
#include "common.cuh"

namespace {

// Largest mesh this entry point accepts; its scratch is one int32 counter per cell plus a control block.
constexpr int64_t NOALLOC_MAX_CELLS = 65536;
constexpr int NOALLOC_CTRL_WORDS = 16;

// scratch: [0, NOALLOC_MAX_CELLS) upwind counters, then the control block:
//   +0 +1 grid barrier (count, generation), +2 error word, +3 largest level, +4 +5 +6 progress flags
//   (one per level modulo 3), +7 cells never reached
static __device__ __align__(256) int32_t g_noalloc_scratch[NOALLOC_MAX_CELLS + NOALLOC_CTRL_WORDS];

// error word value of a face whose cell index is outside [0, n_cells) (after sw::DEV_TIMEOUT, DEV_OVERFLOW)
constexpr int DEV_BAD_INDEX = 3;

// Classification value t = ((nx*Ox) + (ny*Oy)) + (nz*Oz) with separately rounded products and sums.
__device__ __forceinline__ double face_t(const double* n, double ox, double oy, double oz) {
    return __dadd_rn(__dadd_rn(__dmul_rn(n[0], ox), __dmul_rn(n[1], oy)), __dmul_rn(n[2], oz));
}

// One cooperative launch: count upwind cells, then one wavefront per round -- every interior face
// whose upwind cell sits on the current level releases its downwind cell (Alg. 2, one level at a
// time); a counter reaching zero places the cell on the next level.
__global__ void k_levels_noalloc(int64_t N, int64_t F, const int32_t* fc, const double* normal, const uint8_t* flags,
                                 double ox, double oy, double oz, int32_t* level, int32_t* scratch,
                                 long long budget) {
    int32_t* count = scratch;
    int32_t* ctrl = scratch + NOALLOC_MAX_CELLS;
    sw::GridBar* bar = reinterpret_cast<sw::GridBar*>(ctrl);
    int* err = ctrl + 2;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = tid; c < N; c += nth) count[c] = 0;
    if (!sw::grid_sync(bar, gridDim.x, budget, err)) return;
    for (int64_t f = tid; f < F; f += nth) {
        if (flags[f] & (SWEEP_FACE_BOUNDARY | SWEEP_FACE_PERIODIC)) continue;
        const int32_t c0 = fc[2 * f], c1 = fc[2 * f + 1];
        if (c0 < 0 || c0 >= N || c1 < 0 || c1 >= N) {  // the faces are not validated: refuse, touch nothing
            atomicCAS(err, sw::DEV_OK, DEV_BAD_INDEX);
            continue;
        }
        const double t = face_t(normal + 3 * f, ox, oy, oz);
        if (t > 0.0) atomicAdd(&count[c1], 1);
        else if (t < 0.0) atomicAdd(&count[c0], 1);
    }
    // every face the wavefront rounds read was checked above; a bad one ends the launch here
    if (!sw::grid_sync(bar, gridDim.x, budget, err)) return;
    for (int64_t c = tid; c < N; c += nth) level[c] = count[c] == 0 ? 0 : -1;
    if (!sw::grid_sync(bar, gridDim.x, budget, err)) return;
    for (int L = 0;; ++L) {
        // the flag of level L+1 was last read two barriers ago: safe to clear now
        if (tid == 0) ctrl[4 + (L + 1) % 3] = 0;
        for (int64_t f = tid; f < F; f += nth) {
            if (flags[f] & (SWEEP_FACE_BOUNDARY | SWEEP_FACE_PERIODIC)) continue;
            const double t = face_t(normal + 3 * f, ox, oy, oz);
            if (t == 0.0) continue;
            const int32_t up = t > 0.0 ? fc[2 * f] : fc[2 * f + 1];
            const int32_t down = t > 0.0 ? fc[2 * f + 1] : fc[2 * f];
            if (sw::ld_relaxed_i32(&level[up]) != L) continue;  // written by other blocks: read through L2
            if (atomicSub(&count[down], 1) == 1) {
                level[down] = L + 1;
                atomicMax(&ctrl[3], L + 1);
                ctrl[4 + L % 3] = 1;
            }
        }
        if (!sw::grid_sync(bar, gridDim.x, budget, err)) return;
        if (sw::ld_relaxed_i32(&ctrl[4 + L % 3]) == 0) break;
    }
    for (int64_t c = tid; c < N; c += nth)
        if (sw::ld_relaxed_i32(&level[c]) < 0) atomicAdd(&ctrl[7], 1);
}

}  // namespace

extern "C" sweep_status sweep_levels_noalloc(int device, void* cuda_stream, int64_t n_cells, int64_t n_faces,
                                             const int32_t* face_cells, const double* normal, const uint8_t* flags,
                                             const double* omega, int32_t* level, int32_t* depth) {
    if (n_cells < 1 || n_cells > NOALLOC_MAX_CELLS || n_faces < 0) return SWEEP_ERR_INVALID_ARG;
    if (!omega || !level || !depth || (n_faces > 0 && (!face_cells || !normal || !flags))) return SWEEP_ERR_INVALID_ARG;
    if (device < 0) return SWEEP_ERR_INVALID_ARG;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return SWEEP_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return SWEEP_ERR_INVALID_ARG;
    }
    sweep_status rc = SWEEP_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // The device address of the scratch array on this device (its name is only a host-side stand-in).
    // The first call on a device loads the library's device code and looks the address up; later calls
    // look it up again, which allocates nothing and is cheap, so that the address stays right if the
    // device's primary context was destroyed and created again (cudaDeviceReset) in between.
    void* sp = nullptr;
    if (cudaGetSymbolAddress(&sp, g_noalloc_scratch) != cudaSuccess || !sp) {
        cudaGetLastError();
        cudaSetDevice(prev);
        return SWEEP_ERR_CUDA;
    }
    int32_t* scratch = static_cast<int32_t*>(sp);
    int32_t* ctrl = scratch + NOALLOC_MAX_CELLS;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_levels_noalloc, 256, 0);
    if (per_sm < 1) per_sm = 1;
    int blocks = sms * per_sm;
    const int64_t work = n_faces > n_cells ? n_faces : n_cells;
    if ((int64_t)blocks * 256 > work) blocks = (int)((work + 255) / 256);
    if (blocks < 1) blocks = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int32_t h[NOALLOC_CTRL_WORDS];
    cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(int32_t) * NOALLOC_CTRL_WORDS, st);
    if (e == cudaSuccess)
        e = cudaLaunchKernelEx(&cfg, k_levels_noalloc, (int64_t)n_cells, (int64_t)n_faces, face_cells, normal, flags,
                               omega[0], omega[1], omega[2], level, scratch, (long long)(1 << 22));
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, ctrl, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        rc = SWEEP_ERR_CUDA;
    } else if (h[2] == DEV_BAD_INDEX) {
        rc = SWEEP_ERR_INVALID_ARG;
    } else if (h[2] != sw::DEV_OK) {
        rc = SWEEP_ERR_TIMEOUT;
    } else if (h[7] > 0) {
        rc = SWEEP_ERR_CYCLE;
    } else {
        *depth = h[3] + 1;
    }
    cudaSetDevice(prev);
    return rc;
}
