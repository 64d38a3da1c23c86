// Persistent multi-system step: one cooperative launch advances every resident
// system of a batch by n steps of Fig. 1 (arxiv 1804.06205).  The blocks stay
// resident for the whole launch and take the work of each phase in turn --
// beads, cell tiles or pair-kernel bricks, grid-strided -- with a grid-wide
// barrier between phases instead of a kernel boundary.  Each phase calls the
// same device functions as the separate kernels (update_one, scatter_one,
// gather_one, pair_brick, bond_vel_one), so both paths give the same bits.
//
// Every barrier wait is bounded: a block that waits longer than its clock64()
// budget records ST_TIMEOUT in the handle's status and leaves the kernel; the
// other blocks then time out at the same barrier and leave too, and the host
// reports DPD_ETIMEOUT.  Nothing traps or spins without a limit.
#pragma once

#include "kernels.cuh"

namespace dpd {

// The grid barrier's words (device memory, zeroed by the host before each
// launch): blocks arrive on the counter of their group of BAR_GROUP blocks,
// the last arrival of a group on the top counter, and the last arrival there
// advances the generation every waiting block polls.  `work` hands out the
// pair phase's bricks.
constexpr int BAR_GROUP = 32;
constexpr int BAR_MAX_GROUPS = 256;
struct GridBar {
    unsigned int count[BAR_MAX_GROUPS];
    unsigned int top;
    unsigned int gen;
    unsigned int work;
    unsigned int pad;
};

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// All `nblocks` blocks of the grid meet here.  Returns false (in every thread
// of the block) if this block gave up after `budget` clock cycles.
__device__ __forceinline__ bool grid_barrier(GridBar *bar, unsigned int nblocks,
                                             long long budget, int *status) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int g = ld_acquire_gpu(&bar->gen);
        __threadfence();   // this block's writes before its arrival
        const unsigned int grp = blockIdx.x / BAR_GROUP;
        const unsigned int ngroups = (nblocks + BAR_GROUP - 1) / BAR_GROUP;
        const unsigned int gsize = min((unsigned int)BAR_GROUP, nblocks - grp * BAR_GROUP);
        bool released = false;
        if (atomicAdd(&bar->count[grp], 1u) == gsize - 1) {
            // no block of this group can arrive again before the generation moves
            atomicExch(&bar->count[grp], 0u);
            __threadfence();
            if (atomicAdd(&bar->top, 1u) == ngroups - 1) {
                atomicExch(&bar->top, 0u);
                __threadfence();
                atomicAdd(&bar->gen, 1u);   // release every waiting block
                released = true;
            }
        }
        if (!released) {
            const long long t0 = clock64();
            while (ld_acquire_gpu(&bar->gen) == g) {
                if (clock64() - t0 > budget) {
                    atomicOr(status, ST_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Exclusive scan of one value per thread over a block of NT threads.
template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan_nt(uint32_t v, uint32_t *total) {
    __shared__ uint32_t s_w[NT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t inc = warp_incl_scan(v);
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const uint32_t w = lane < NT / 32 ? s_w[lane] : 0u;
        const uint32_t wi = warp_incl_scan(w);
        if (lane < NT / 32) s_w[lane] = wi - w;
        if (lane == NT / 32 - 1) *total = wi;
    }
    __syncthreads();
    const uint32_t r = s_w[wid] + inc - v;
    __syncthreads();
    return r;
}

// Tile `tile` (SCAN_B cells) of the counting sort's scan, as k_scan1 / k_scan3b
// with NT threads per block: the tile's total, then its exclusive starts.
template <int NT>
__device__ __forceinline__ void scan_tile_sum(const uint32_t *count, int ncell, uint32_t *bsum,
                                              int tile) {
    constexpr int V = SCAN_B / NT;
    __shared__ uint32_t tot;
    const int base = tile * SCAN_B + threadIdx.x * V;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < V; ++k)
        if (base + k < ncell) s += count[base + k];
    block_excl_scan_nt<NT>(s, &tot);
    if (threadIdx.x == 0) bsum[tile] = tot;
}

template <int NT>
__device__ __forceinline__ void scan_tile_final(uint32_t *count, int ncell, const uint32_t *bsum,
                                                uint32_t *cell_start, int tile, int ntiles) {
    constexpr int V = SCAN_B / NT;
    __shared__ uint32_t tot;
    uint32_t before = 0;
    for (int j = threadIdx.x; j < tile; j += NT) before += bsum[j];
    block_excl_scan_nt<NT>(before, &tot);
    before = tot;
    const int b0 = tile * SCAN_B + threadIdx.x * V;
    uint32_t v[V];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < V; ++k) {
        v[k] = (b0 + k < ncell) ? count[b0 + k] : 0u;
        sum += v[k];
    }
    uint32_t run = block_excl_scan_nt<NT>(sum, &tot) + before;
#pragma unroll
    for (int k = 0; k < V; ++k)
        if (b0 + k < ncell) {
            cell_start[b0 + k] = run;
            run += v[k];
            count[b0 + k] = 0u;
        }
    if (tile == ntiles - 1 && threadIdx.x == NT - 1) cell_start[ncell] = run;
}

// Everything one launch needs; [2] entries are indexed by the parity of the
// step (the ping-pong buffers of v, f and ids swap every step).
template <class P>
struct StepArgs {
    int nsteps, nbeads, ncells, nbricks, ntiles;
    int with_update;                 // the first step starts with the position update
    UpdArgs<P> upd;
    ScatterArgs<P> sc[2];
    GatherArgs<P> ga[2];
    PairLaunch<P> pl[2];             // [p].fpair: that step's force buffer
    BondArgs<P> bo[2];
    uint32_t *count, *bsum, *cell_start;
    GridBar *bar;
    long long budget;                // clock cycles a block may wait at one barrier
    int *status;
};

template <class P, int T>
__global__ void __launch_bounds__(T, P::kOffsets ? PAIR_THREADS_PER_SM / T : 1)
    k_steps(StepArgs<P> a) {
    griddep_wait();
    const unsigned int nb = gridDim.x;
    const int gstride = (int)(gridDim.x * T);
    const int gt = (int)(blockIdx.x * T + threadIdx.x);
    auto sync = [&]() { return grid_barrier(a.bar, nb, a.budget, a.status); };
    if (a.with_update) {
        for (int t = gt; t < a.nbeads; t += gstride) update_one<P>(a.upd, t);
        if (!sync()) return;
    }
    for (int k = 0; k < a.nsteps; ++k) {
        const int p = k & 1;
        for (int tile = blockIdx.x; tile < a.ntiles; tile += nb)
            scan_tile_sum<T>(a.count, a.ncells, a.bsum, tile);
        if (!sync()) return;
        for (int tile = blockIdx.x; tile < a.ntiles; tile += nb)
            scan_tile_final<T>(a.count, a.ncells, a.bsum, a.cell_start, tile, a.ntiles);
        if (!sync()) return;
        for (int t = gt; t < a.nbeads; t += gstride) scatter_one<P>(a.sc[p], t);
        if (!sync()) return;
        for (int t = gt; t < a.nbeads; t += gstride) gather_one<P, false>(a.ga[p], t);
        if (!sync()) return;
        {   // bricks handed out one at a time (their costs vary with occupancy);
            // the tickets of step k are [k (nbricks + nb), (k + 1) (nbricks + nb)):
            // every brick once, then one ticket per block that finds none left
            __shared__ int s_br;
            const unsigned int base = (unsigned int)k * (unsigned int)(a.nbricks + (int)nb);
            for (;;) {
                if (threadIdx.x == 0) s_br = (int)(atomicAdd(&a.bar->work, 1u) - base);
                __syncthreads();
                const int br = s_br;
                __syncthreads();
                if (br >= a.nbricks) break;
                if (!pair_brick<P, T, false, true>(a.pl[p], br)) return;   // ST_TIMEOUT is set
            }
        }
        if (!sync()) return;
        // bonds and velocity; every step but the last also makes the next
        // step's position update
        if (k + 1 < a.nsteps) {
            for (int t = gt; t < a.nbeads; t += gstride)
                bond_vel_one<P, false, false, true>(a.bo[p], t);
        } else {
            for (int t = gt; t < a.nbeads; t += gstride)
                bond_vel_one<P, false, false, false>(a.bo[p], t);
        }
        if (k + 1 < a.nsteps && !sync()) return;
    }
}

// Check of the failure detection on the grid barrier, without a fault: the
// grid waits at one barrier that expects `expect` blocks.  With expect equal
// to the grid, the barrier completes; with one more, nobody can complete it,
// every block gives up after `budget` cycles and records ST_TIMEOUT.
static __global__ void k_grid_wait_check(GridBar *bar, unsigned int expect, long long budget,
                                         int *status) {
    grid_barrier(bar, expect, budget, status);
}

}  // namespace dpd
