// dpd_cells_noalloc: the cell division of the engine (periodic wrap, cell
// key, canonical (cell, id) counting sort) for positions that are already in
// device memory, in a form that allocates no memory at all.
//
// Who needs it: callers that cannot call cudaMalloc -- code whose device
// memory is all owned by a framework's caching allocator or by a fixed arena
// budgeted up front (a serving process must not grow its footprint behind
// the allocator's back), and code that must not hit cudaMalloc's implicit
// device synchronisation.  They pass every input and output buffer; the only
// extra memory is the fixed scratch array below.
//
// The scratch is one file-scope __device__ array of DPD_NOALLOC_MAX_N + 2050
// 32-bit words (16 MiB + 8 KiB).  Every GPU that loads this code holds it until
// the process exits.  Host code cannot use the array's name as a device
// address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it.  All calls
// share the array and it keeps the last call's contents; calls that overlap
// on the GPU (two streams, or two host threads) race on it.
//
// Steps: wrap + key + arrival rank (atomics on the counts), exclusive scan of
// the counts, arrival-order scatter, then every bead finds its canonical slot
// by counting the smaller ids of its cell (k loads for a cell of k beads, done
// by all of them in parallel) and places itself there.
#include <cuda_runtime.h>

#include <mutex>

#include "dpd.h"
#include "kernels.cuh"

namespace {

constexpr int64_t kNaBsumWords = DPD_NOALLOC_MAX_CELLS / dpd::SCAN_B + 2;
constexpr int64_t kNaWords = DPD_NOALLOC_MAX_N + kNaBsumWords;

// arrival rank of every bead in its cell, then the scan's block sums
static __device__ __align__(256) uint32_t g_na_scratch[kNaWords];

constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
uint32_t *g_na_ptr[kMaxDevices] = {nullptr};

// The device address of g_na_scratch on the current device (looked up once).
cudaError_t scratch_ptr(uint32_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

// wrap, key, arrival rank (the counts accumulate in cell_start, zeroed first)
__global__ void __launch_bounds__(256) k_na_keys(int n, dpd::Geo g, const double *pos,
                                                 uint32_t *key, uint32_t *count, uint32_t *rank) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = dpd::wrap_exact(pos[3 * i], g.L[0]);
    const double y = dpd::wrap_exact(pos[3 * i + 1], g.L[1]);
    const double z = dpd::wrap_exact(pos[3 * i + 2], g.L[2]);
    const uint32_t cx = (uint32_t)dpd::cell_of(x, g.inv_h[0], g.nx);
    const uint32_t cy = (uint32_t)dpd::cell_of(y, g.inv_h[1], g.ny);
    const uint32_t cz = (uint32_t)dpd::cell_of(z, g.inv_h[2], g.nz);
    const uint32_t k = (cz * (uint32_t)g.ny + cy) * (uint32_t)g.nx + cx;
    key[i] = k;
    rank[i] = atomicAdd(&count[k], 1u);
}

// in-place block scan: counts in, exclusive starts out
__global__ void __launch_bounds__(dpd::SCAN_T) k_na_scan3(uint32_t *cs, int ncell,
                                                          const uint32_t *bsum) {
    const int base = blockIdx.x * dpd::SCAN_B + threadIdx.x * dpd::SCAN_V;
    uint32_t v[dpd::SCAN_V];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < dpd::SCAN_V; ++k) {
        v[k] = (base + k < ncell) ? cs[base + k] : 0u;
        s += v[k];
    }
    __shared__ uint32_t tot;
    uint32_t run = dpd::block_excl_scan(s, &tot) + bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < dpd::SCAN_V; ++k)
        if (base + k < ncell) {
            cs[base + k] = run;
            run += v[k];
        }
}

// arrival order: order[cell start + arrival rank] = id
__global__ void __launch_bounds__(256) k_na_scatter(int n, const uint32_t *key,
                                                    const uint32_t *rank, const uint32_t *cs,
                                                    int32_t *order) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    order[cs[key[i]] + rank[i]] = i;
}

// Canonical slot of every bead: its cell's start plus the number of the
// cell's ids below its own (the cell's ids in arrival order are in `order`).
// Every bead counts in parallel, so a cell of k beads costs k loads per bead;
// slot[] reuses the arrival-rank words, which nothing reads any more.
__global__ void __launch_bounds__(256) k_na_rank(int n, const uint32_t *key, const uint32_t *cs,
                                                 const int32_t *order, uint32_t *slot) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = key[i];
    const int b = (int)cs[k], e = (int)cs[k + 1];
    int u = b;
    for (int q = b; q < e; ++q) u += order[q] < i;
    slot[i] = (uint32_t)u;
}

__global__ void __launch_bounds__(256) k_na_place(int n, const uint32_t *slot, int32_t *order) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    order[slot[i]] = i;
}

}  // namespace

extern "C" int dpd_cells_noalloc(const double *pos_dev, int64_t n, const dpd_box *box,
                                 uint32_t *key_dev, int32_t *order_dev,
                                 uint32_t *cell_start_dev, void *cuda_stream) {
    if (!pos_dev || !box || !key_dev || !order_dev || !cell_start_dev) return DPD_EINVAL;
    if (n <= 0 || n > DPD_NOALLOC_MAX_N) return DPD_EINVAL;
    dpd::Geo g{};
    int64_t ncell = 1;
    int nc[3];
    for (int k = 0; k < 3; ++k) {
        const double L = box->L[k];
        if (!(L >= 3.0) || !(L < 1e300)) return DPD_EINVAL;
        const double f = floor(L);
        if (f > (double)DPD_NOALLOC_MAX_CELLS) return DPD_EINVAL;
        nc[k] = (int)f;
        g.L[k] = L;
        g.h[k] = L / f;
        g.inv_h[k] = f / L;
        // checked after every factor, so the product stays below 2^44 and the
        // scan's block sums (sized for DPD_NOALLOC_MAX_CELLS) always suffice
        ncell *= (int64_t)nc[k];
        if (ncell > DPD_NOALLOC_MAX_CELLS) return DPD_EINVAL;
    }
    g.nx = nc[0];
    g.ny = nc[1];
    g.nz = nc[2];
    g.ncell = (int)ncell;
    uint32_t *scratch = nullptr;
    if (scratch_ptr(&scratch) != cudaSuccess) return DPD_ECUDA;
    uint32_t *rank = scratch;
    uint32_t *bsum = scratch + DPD_NOALLOC_MAX_N;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int C = (int)ncell, N = (int)n;
    const int nb = (C + dpd::SCAN_B - 1) / dpd::SCAN_B;
    // the counts accumulate in cell_start, which must start at zero
    if (cudaMemsetAsync(cell_start_dev, 0, (size_t)(C + 1) * sizeof(uint32_t), st) != cudaSuccess)
        return DPD_ECUDA;
    // the arrival ranks are all written before they are read
    k_na_keys<<<(N + 255) / 256, 256, 0, st>>>(N, g, pos_dev, key_dev, cell_start_dev, rank);
    dpd::k_scan1<<<nb, dpd::SCAN_T, 0, st>>>(cell_start_dev, C, bsum);
    dpd::k_scan2<<<1, dpd::SCAN_T, 0, st>>>(bsum, nb, cell_start_dev, C);
    k_na_scan3<<<nb, dpd::SCAN_T, 0, st>>>(cell_start_dev, C, bsum);
    k_na_scatter<<<(N + 255) / 256, 256, 0, st>>>(N, key_dev, rank, cell_start_dev, order_dev);
    k_na_rank<<<(N + 255) / 256, 256, 0, st>>>(N, key_dev, cell_start_dev, order_dev, rank);
    k_na_place<<<(N + 255) / 256, 256, 0, st>>>(N, rank, order_dev);
    return cudaGetLastError() == cudaSuccess ? DPD_OK : DPD_ECUDA;
}
