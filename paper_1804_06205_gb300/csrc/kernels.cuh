// Device code of the DPD step loop (arxiv 1804.06205, Fig. 1) for sm_103a and
// the per-precision engine that sequences it.  Included by engine_f32.cu and
// engine_f64.cu, each of which instantiates one precision.
//
// One step (Fig. 1), all on the device:
//   k_update      1.-2. r += dt v + dt^2/2 f, periodic wrap in FP64, new cell
//                 key, histogram of cell occupancy (atomics on counts)
//   k_scan*       3.    exclusive scan of the counts -> cell_start
//   k_scatter     3.    slot = cell_start[key] + arrival rank
//   k_cellfix     3.    canonical (cell, id) order inside each cell
//   k_gather      3.    permute the state into the new order, v~ = v + lambda dt f
//   k_pair        4.    eq. 3-4 + dissipative/random pair terms, 27-cell full shell
//   k_bond_vel    4.-5. eqs. 6-8 bonded terms, then v += dt/2 (f + f')
//   k_reduce*           FP64 sums for the observables (sampled steps only)
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "engine.h"

namespace dpd {

// --------------------------------------------------------------------------
// Precision policies.
//   PF32: positions are FP32 offsets inside the bead's cell (x = c h + o),
//         forces and velocities FP32.
//   PF64: positions are absolute FP64 coordinates, everything FP64.
// Element w of a position holds the bead type (a small integer value); w of
// v~ holds the bead id (bit pattern).
// --------------------------------------------------------------------------
struct __align__(32) dvec4 {
    double x, y, z, w;
};

struct PF32 {
    using real = float;
    using vec4 = float4;
    static constexpr bool kOffsets = true;
    static __device__ __forceinline__ real pack_id(int32_t i) { return __int_as_float(i); }
    static __device__ __forceinline__ int32_t unpack_id(real w) { return __float_as_int(w); }
};

struct PF64 {
    using real = double;
    using vec4 = dvec4;
    static constexpr bool kOffsets = false;
    static __device__ __forceinline__ real pack_id(int32_t i) {
        return __longlong_as_double((long long)i);
    }
    static __device__ __forceinline__ int32_t unpack_id(real w) {
        return (int32_t)__double_as_longlong(w);
    }
};

template <class V, class R>
__device__ __forceinline__ V mk4(R x, R y, R z, R w) {
    V v;
    v.x = x; v.y = y; v.z = z; v.w = w;
    return v;
}

// Device status bits (sticky until the handle is destroyed).
enum : int { ST_NONFINITE = 1, ST_TIMEOUT = 2, ST_BADINPUT = 4 };

// --------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the
// published round function: two 32x32->64 products of counter words 0 and 2
// with the published multipliers, high halves mixed with the other two words
// and the round key, key advanced by the published Weyl increments.
// --------------------------------------------------------------------------
__device__ __forceinline__ uint2 philox_xy(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                           uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return make_uint2(c0, c1);   // outputs 0 and 1 (2 and 3 are not needed)
}

// Uniform (2*(x>>9)+1) * 2^-24 in (0, 1), exact in binary32.
__device__ __forceinline__ float u01_f32(uint32_t x) {
    return __uint2float_rn((x >> 8) | 1u) * 0x1p-24f;
}
__device__ __forceinline__ double u01_f64(uint32_t x) {
    return (double)((x >> 8) | 1u) * 0x1p-24;
}

__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }

// theta from Box-Muller on outputs 0 and 1 (noise 0) or sqrt(3)(2u-1) (noise 1).
__device__ __forceinline__ float theta_of(uint2 x, int noise, float) {
    const float u0 = u01_f32(x.x);
    if (noise) return 1.7320508075688772f * (2.0f * u0 - 1.0f);
    const float u1 = u01_f32(x.y);
    return sqrtf(-2.0f * logf(u0)) * cospif(2.0f * u1);
}
__device__ __forceinline__ double theta_of(uint2 x, int noise, double) {
    const double u0 = u01_f64(x.x);
    if (noise) return 1.7320508075688772 * (2.0 * u0 - 1.0);
    const double u1 = u01_f64(x.y);
    return sqrt(-2.0 * log(u0)) * cospi(2.0 * u1);
}

// --------------------------------------------------------------------------
// Periodic wrap and cell key, FP64, with no fused multiply-add so that the
// result is the IEEE value of x - L*floor(x/L) and floor(x * inv_h).
// --------------------------------------------------------------------------
__device__ __forceinline__ double wrap_exact(double x, double L) {
    const double q = floor(__ddiv_rn(x, L));
    double y = __dsub_rn(x, __dmul_rn(L, q));
    if (y < 0.0) y = __dadd_rn(y, L);
    if (y >= L) y = __dsub_rn(y, L);
    return y;
}
__device__ __forceinline__ int cell_of(double x, double inv_h, int n) {
    const double q = floor(__dmul_rn(x, inv_h));
    return (q > 0.0) ? (q < (double)(n - 1) ? (int)q : n - 1) : 0;   // NaN -> 0
}

struct Geo {
    int nx, ny, nz, ncell;
    double L[3], h[3], inv_h[3];
};

__device__ __forceinline__ void decode_key(uint32_t k, const Geo &g, int &cx, int &cy, int &cz) {
    cx = (int)(k % (uint32_t)g.nx);
    const uint32_t q = k / (uint32_t)g.nx;
    cy = (int)(q % (uint32_t)g.ny);
    cz = (int)(q / (uint32_t)g.ny);
}

// --------------------------------------------------------------------------
// a1-a2: position update, wrap, key (and set_state's initial binning).
// --------------------------------------------------------------------------
template <class P>
struct UpdArgs {
    using vec4 = typename P::vec4;
    using real = typename P::real;
    int n;
    Geo g;
    real dt, half_dt2;
    const uint32_t *key;
    const vec4 *pos, *vel, *frc;
    vec4 *pos_tmp;
    uint32_t *key_tmp, *rank, *count;
    long long *counter;
    int *status;
};

template <class P>
__device__ __forceinline__ void place_bead(const Geo &g, double x, double y, double z,
                                           typename P::real type, typename P::vec4 &out,
                                           uint32_t &key, int *status, int bad_bit) {
    using real = typename P::real;
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) atomicOr(status, bad_bit);
    x = wrap_exact(x, g.L[0]);
    y = wrap_exact(y, g.L[1]);
    z = wrap_exact(z, g.L[2]);
    const int cx = cell_of(x, g.inv_h[0], g.nx);
    const int cy = cell_of(y, g.inv_h[1], g.ny);
    const int cz = cell_of(z, g.inv_h[2], g.nz);
    key = ((uint32_t)cz * (uint32_t)g.ny + (uint32_t)cy) * (uint32_t)g.nx + (uint32_t)cx;
    if (P::kOffsets) {
        out = mk4<typename P::vec4, real>((real)(x - (double)cx * g.h[0]),
                                          (real)(y - (double)cy * g.h[1]),
                                          (real)(z - (double)cz * g.h[2]), type);
    } else {
        out = mk4<typename P::vec4, real>((real)x, (real)y, (real)z, type);
    }
}

template <class P>
__global__ void __launch_bounds__(256) k_update(UpdArgs<P> a) {
    using real = typename P::real;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) *a.counter += 1;   // evaluation counter of this step's force
    if (t >= a.n) return;
    const typename P::vec4 p = a.pos[t], v = a.vel[t], f = a.frc[t];
    const real ddx = a.dt * v.x + a.half_dt2 * f.x;
    const real ddy = a.dt * v.y + a.half_dt2 * f.y;
    const real ddz = a.dt * v.z + a.half_dt2 * f.z;
    double x, y, z;
    if (P::kOffsets) {
        int cx, cy, cz;
        decode_key(a.key[t], a.g, cx, cy, cz);
        x = (double)cx * a.g.h[0] + (double)p.x;
        y = (double)cy * a.g.h[1] + (double)p.y;
        z = (double)cz * a.g.h[2] + (double)p.z;
    } else {
        x = (double)p.x; y = (double)p.y; z = (double)p.z;
    }
    typename P::vec4 out;
    uint32_t key;
    place_bead<P>(a.g, x + (double)ddx, y + (double)ddy, z + (double)ddz, p.w, out, key, a.status,
                  ST_NONFINITE);
    a.pos_tmp[t] = out;
    a.key_tmp[t] = key;
    a.rank[t] = atomicAdd(&a.count[key], 1u);
}

template <class P>
struct InitArgs {
    using vec4 = typename P::vec4;
    int n;
    Geo g;
    const double *pos_in, *vel_in;   // [n*3] bead-id order
    const int32_t *types;
    vec4 *pos_tmp, *vel, *frc;
    uint32_t *key_tmp, *rank, *count;
    int32_t *id;
    int *status;
};

template <class P>
__global__ void __launch_bounds__(256) k_init(InitArgs<P> a) {
    using real = typename P::real;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    typename P::vec4 out;
    uint32_t key;
    place_bead<P>(a.g, a.pos_in[3 * i], a.pos_in[3 * i + 1], a.pos_in[3 * i + 2],
                  (real)a.types[i], out, key, a.status, ST_BADINPUT);
    a.pos_tmp[i] = out;
    a.key_tmp[i] = key;
    a.rank[i] = atomicAdd(&a.count[key], 1u);
    const double vx = a.vel_in[3 * i], vy = a.vel_in[3 * i + 1], vz = a.vel_in[3 * i + 2];
    if (!(isfinite(vx) && isfinite(vy) && isfinite(vz))) atomicOr(a.status, ST_BADINPUT);
    a.vel[i] = mk4<typename P::vec4, real>((real)vx, (real)vy, (real)vz, (real)0);
    a.frc[i] = mk4<typename P::vec4, real>((real)0, (real)0, (real)0, (real)0);
    a.id[i] = i;
}

// --------------------------------------------------------------------------
// a3: counting sort.  Exclusive scan of the per-cell counts in three passes
// (block sums, scan of block sums, block scans plus offsets); the third pass
// also clears the counts for the next step.
// --------------------------------------------------------------------------
constexpr int SCAN_T = 256, SCAN_V = 8, SCAN_B = SCAN_T * SCAN_V;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive block scan of one value per thread (blockDim.x == SCAN_T).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t s_w[SCAN_T / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t inc = warp_incl_scan(v);
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < SCAN_T / 32 ? s_w[lane] : 0u;
        const uint32_t wi = warp_incl_scan(w);
        if (lane < SCAN_T / 32) s_w[lane] = wi - w;
        if (lane == SCAN_T / 32 - 1) *total = wi;
    }
    __syncthreads();
    const uint32_t r = s_w[wid] + inc - v;
    __syncthreads();
    return r;
}

static __global__ void __launch_bounds__(SCAN_T) k_scan1(const uint32_t *count, int ncell,
                                                  uint32_t *bsum) {
    const int base = blockIdx.x * SCAN_B + threadIdx.x * SCAN_V;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_V; ++k)
        if (base + k < ncell) s += count[base + k];
    __shared__ uint32_t tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

static __global__ void __launch_bounds__(SCAN_T) k_scan2(uint32_t *bsum, int nb, uint32_t *cell_start,
                                                  int ncell) {
    __shared__ uint32_t tot;
    uint32_t carry = 0;
    for (int b0 = 0; b0 < nb; b0 += SCAN_T) {
        const int b = b0 + threadIdx.x;
        const uint32_t v = b < nb ? bsum[b] : 0u;
        const uint32_t ex = block_excl_scan(v, &tot);
        if (b < nb) bsum[b] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) cell_start[ncell] = carry;
}

static __global__ void __launch_bounds__(SCAN_T) k_scan3(uint32_t *count, int ncell,
                                                  const uint32_t *bsum, uint32_t *cell_start) {
    const int base = blockIdx.x * SCAN_B + threadIdx.x * SCAN_V;
    uint32_t v[SCAN_V];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_V; ++k) {
        v[k] = (base + k < ncell) ? count[base + k] : 0u;
        s += v[k];
    }
    __shared__ uint32_t tot;
    uint32_t run = block_excl_scan(s, &tot) + bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_V; ++k)
        if (base + k < ncell) {
            cell_start[base + k] = run;
            run += v[k];
            count[base + k] = 0u;
        }
}

static __global__ void __launch_bounds__(256) k_scatter(int n, const uint32_t *key_tmp,
                                                 const uint32_t *rank, const uint32_t *cell_start,
                                                 const int32_t *id_old, uint32_t *src,
                                                 int32_t *sid) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint32_t slot = cell_start[key_tmp[t]] + rank[t];
    src[slot] = (uint32_t)t;
    sid[slot] = id_old[t];
}

// Atomic ranks give an arbitrary order inside a cell; sort each cell's
// entries by bead id (cells hold ~3 beads: insertion sort).
static __global__ void __launch_bounds__(256) k_cellfix(int ncell, const uint32_t *cell_start,
                                                 uint32_t *src, int32_t *sid) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int b = (int)cell_start[c], e = (int)cell_start[c + 1];
    for (int i = b + 1; i < e; ++i) {
        const int32_t ki = sid[i];
        const uint32_t si = src[i];
        int j = i - 1;
        while (j >= b && sid[j] > ki) {
            sid[j + 1] = sid[j];
            src[j + 1] = src[j];
            --j;
        }
        sid[j + 1] = ki;
        src[j + 1] = si;
    }
}

template <class P>
struct GatherArgs {
    using vec4 = typename P::vec4;
    using real = typename P::real;
    int n;
    real lam_dt;
    const uint32_t *src;
    const int32_t *sid;
    const vec4 *pos_tmp, *vel_old, *frc_old;
    const uint32_t *key_tmp;
    vec4 *pos, *vel, *frc, *vt;
    uint32_t *key;
    int32_t *id, *inv_perm;
};

template <class P>
__global__ void __launch_bounds__(256) k_gather(GatherArgs<P> a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n) return;
    const uint32_t s = a.src[t];
    const int32_t i = a.sid[t];
    const typename P::vec4 v = a.vel_old[s], f = a.frc_old[s];
    a.pos[t] = a.pos_tmp[s];
    a.key[t] = a.key_tmp[s];
    a.vel[t] = v;
    a.frc[t] = f;
    a.id[t] = i;
    a.inv_perm[i] = t;
    // Fig. 1 step 2: velocity predictor used by the dissipative force
    a.vt[t] = mk4<typename P::vec4, typename P::real>(v.x + a.lam_dt * f.x, v.y + a.lam_dt * f.y,
                                                      v.z + a.lam_dt * f.z, P::pack_id(i));
}

// --------------------------------------------------------------------------
// a4-a5: pair forces, 27-cell full shell (each bead summed by one thread, no
// force atomics).  A block owns a run of X consecutive cells of one x-row.
// It stages the 9 neighbouring row runs (X+2 cells each, periodic) into
// shared memory, then every thread takes one home bead: it walks the 27
// neighbour cells in fixed (dz, dy, dx) order, collects the hits r < 1 in a
// per-thread list and evaluates them in that order.  The neighbour cell's
// periodic shift is applied to the home bead once per cell, so the staged
// records are raw copies and a bead's sum does not depend on the tiling.
// Oversized neighbourhoods are staged in chunks and long hit lists are
// evaluated in passes; both keep the summation order.
// --------------------------------------------------------------------------
template <class P>
struct PairArgs {
    using vec4 = typename P::vec4;
    using real = typename P::real;
    const vec4 *pos, *vt;
    const uint32_t *key, *cell_start;
    vec4 *fpair, *ev;
    const real *a;
    int ntypes;
    int nx, ny, nz;
    int X, segs_per_row;
    real h[3], L[3];
    real gamma, sig_sqdt;
    uint32_t key0, key1;
    int noise;
    const long long *counter;
    int cap, hmax;
};

constexpr int PAIR_MAXX = 64;          // largest tile (cells per block)
constexpr int PAIR_MAXT = 16;          // largest number of bead types

template <class P>
struct PairSmem {
    static size_t bytes(int cap, int X, int T, int hmax) {
        size_t b = 2 * (size_t)cap * sizeof(typename P::vec4);
        b += 9 * (size_t)(X + 3) * sizeof(int);
        b += 27 * 3 * sizeof(int);
        b = (b + 15) & ~(size_t)15;
        b += PAIR_MAXT * PAIR_MAXT * sizeof(typename P::real);
        b += (size_t)hmax * T * sizeof(uint16_t);
        return b;
    }
};

template <class P>
__device__ __forceinline__ void cell_shift(const PairArgs<P> &a, int ci, int cx, int cy, int cz,
                                           typename P::real &sx, typename P::real &sy,
                                           typename P::real &sz) {
    using real = typename P::real;
    const int rr = ci / 3;
    const int ddx = ci - 3 * rr - 1, ddy = rr % 3 - 1, ddz = rr / 3 - 1;
    if (P::kOffsets) {
        // home-bead offset minus the neighbour cell's origin relative to its own cell
        sx = -(real)ddx * a.h[0];
        sy = -(real)ddy * a.h[1];
        sz = -(real)ddz * a.h[2];
    } else {
        // absolute coordinates: undo the periodic wrap of the neighbour cell
        const int ux = cx + ddx, uy = cy + ddy, uz = cz + ddz;
        sx = ux < 0 ? a.L[0] : (ux >= a.nx ? -a.L[0] : (real)0);
        sy = uy < 0 ? a.L[1] : (uy >= a.ny ? -a.L[1] : (real)0);
        sz = uz < 0 ? a.L[2] : (uz >= a.nz ? -a.L[2] : (real)0);
    }
}

template <class P, int T, bool SAMPLE>
__global__ void __launch_bounds__(T) k_pair(PairArgs<P> a) {
    using real = typename P::real;
    using vec4 = typename P::vec4;
    extern __shared__ __align__(32) unsigned char smem[];
    const int cap = a.cap;
    const int X = a.X;
    vec4 *s_pos = reinterpret_cast<vec4 *>(smem);
    vec4 *s_vt = s_pos + cap;
    int *s_cs = reinterpret_cast<int *>(s_vt + cap);
    int *s_pc = s_cs + 9 * (X + 3);                         // pieces: src, dst, len
    size_t off = (size_t)((unsigned char *)(s_pc + 81) - smem);
    off = (off + 15) & ~(size_t)15;
    real *s_a = reinterpret_cast<real *>(smem + off);
    uint16_t *s_hit = reinterpret_cast<uint16_t *>(s_a + PAIR_MAXT * PAIR_MAXT);

    const int tid = threadIdx.x;
    const int seg = blockIdx.x;
    const int row = seg / a.segs_per_row;
    const int x0 = (seg - row * a.segs_per_row) * X;
    const int cy = row % a.ny, cz = row / a.ny;
    const int Xe = min(X, a.nx - x0);
    const int W = Xe + 3;

    for (int e = tid; e < a.ntypes * a.ntypes; e += T) s_a[e] = a.a[e];
    // per staged cell: counts (k = 0..Xe+1 <-> ux = -1..Xe), k = Xe+2 is the row end
    for (int e = tid; e < 9 * W; e += T) {
        const int r = e / W, k = e - r * W;
        int cnt = 0;
        if (k <= Xe + 1) {
            const int yy = (cy + (r % 3) - 1 + a.ny) % a.ny;
            const int zz = (cz + (r / 3) - 1 + a.nz) % a.nz;
            const int xx = (x0 + k - 1 + a.nx) % a.nx;
            const uint32_t key = ((uint32_t)zz * a.ny + yy) * a.nx + xx;
            cnt = (int)(a.cell_start[key + 1] - a.cell_start[key]);
        }
        s_cs[e] = cnt;
    }
    __syncthreads();
    if (tid < 32) {   // exclusive scan of the 9*W counts: staged start of each cell
        int carry = 0;
        for (int b = 0; b < 9 * W; b += 32) {
            const int v = (b + tid < 9 * W) ? s_cs[b + tid] : 0;
            int inc = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, inc, o);
                if (tid >= o) inc += u;
            }
            if (b + tid < 9 * W) s_cs[b + tid] = carry + inc - v;
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
    }
    __syncthreads();
    if (tid < 9) {    // contiguous source runs of each staged row (split at x wraps)
        const int r = tid;
        const int yy = (cy + (r % 3) - 1 + a.ny) % a.ny;
        const int zz = (cz + (r / 3) - 1 + a.nz) % a.nz;
        const uint32_t rowkey = ((uint32_t)zz * a.ny + yy) * a.nx;
        int np = 0, kfirst = 0;
        for (int k = 1; k <= Xe + 2; ++k) {
            const bool end = (k == Xe + 2) || ((x0 + k - 1 + a.nx) % a.nx == 0);
            if (end) {
                const int xx = (x0 + kfirst - 1 + a.nx) % a.nx;
                s_pc[r * 9 + np * 3 + 0] = (int)a.cell_start[rowkey + xx];
                s_pc[r * 9 + np * 3 + 1] = s_cs[r * W + kfirst];
                s_pc[r * 9 + np * 3 + 2] = s_cs[r * W + k] - s_cs[r * W + kfirst];
                ++np;
                kfirst = k;
            }
        }
        for (; np < 3; ++np) s_pc[r * 9 + np * 3 + 2] = 0;
    }
    __syncthreads();

    const int S = s_cs[9 * W - 1];                       // staged beads in total
    const int hb_lo = s_cs[4 * W + 1], hb_hi = s_cs[4 * W + Xe + 1];
    const int H = hb_hi - hb_lo;
    const int gbase = (int)a.cell_start[((uint32_t)cz * a.ny + cy) * a.nx + x0];
    const long long sctr = *a.counter;
    const uint32_t s_lo = (uint32_t)(unsigned long long)sctr;
    const uint32_t s_hi = (uint32_t)((unsigned long long)sctr >> 32);
    const int nt = a.ntypes;
    const int hmax = a.hmax;
    int staged_lo = -1;

    for (int hb0 = 0; hb0 < H; hb0 += T) {
        const int hb = hb0 + tid;
        const bool active = hb < H;
        const int g = gbase + (active ? hb : 0);
        vec4 pi = a.pos[g], vi = a.vt[g];
        int cxi = 0, cyi = cy, czi = cz, uxi = 0;
        if (active) {
            cxi = (int)(a.key[g] % (uint32_t)a.nx);
            uxi = cxi - x0;
        }
        const int ti = (int)pi.w;
        const int32_t idi = P::unpack_id(vi.w);
        real fx = 0, fy = 0, fz = 0, wc = 0, ep = 0;

        for (int c0 = 0; c0 < S; c0 += cap) {
            const int c1 = min(S, c0 + cap);
            if (staged_lo != c0) {
                __syncthreads();   // everyone is done with the previous chunk
                const int wid = tid >> 5, lane = tid & 31;
                for (int pc = wid; pc < 27; pc += T / 32) {
                    const int src = s_pc[pc * 3], dst = s_pc[pc * 3 + 1], len = s_pc[pc * 3 + 2];
                    const int lo = max(dst, c0), hi = min(dst + len, c1);
                    for (int q = lo + lane; q < hi; q += 32) {
                        s_pos[q - c0] = a.pos[src + (q - dst)];
                        s_vt[q - c0] = a.vt[src + (q - dst)];
                    }
                }
                staged_lo = c0;
                __syncthreads();
            }
            if (!active) continue;
            int ci = 0, q = 0;
            bool more = true;
            while (more) {
                // scan: collect up to hmax hits in (cell, slot) order
                int nh = 0;
                more = false;
                for (; ci < 27; ++ci) {
                    const int rr = ci / 3;
                    const int k = uxi + (ci - 3 * rr);
                    const int qb = max(s_cs[rr * W + k], c0);
                    const int qe = min(s_cs[rr * W + k + 1], c1);
                    if (q < qb) q = qb;
                    if (q >= qe) continue;
                    real sx, sy, sz;
                    cell_shift<P>(a, ci, cxi, cyi, czi, sx, sy, sz);
                    const real bx = pi.x + sx, by = pi.y + sy, bz = pi.z + sz;
                    for (; q < qe; ++q) {
                        const vec4 pj = s_pos[q - c0];
                        const real dx = bx - pj.x, dy = by - pj.y, dz = bz - pj.z;
                        const real r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 < (real)1 && r2 > (real)0) {
                            s_hit[nh * T + tid] = (uint16_t)(((q - c0) << 5) | ci);
                            if (++nh == hmax) break;
                        }
                    }
                    if (nh == hmax) {
                        ++q;
                        more = true;
                        break;
                    }
                }
                // evaluate the hits in order
                for (int m = 0; m < nh; ++m) {
                    const int e = s_hit[m * T + tid];
                    const int jl = e >> 5, cj = e & 31;
                    real sx, sy, sz;
                    cell_shift<P>(a, cj, cxi, cyi, czi, sx, sy, sz);
                    const vec4 pj = s_pos[jl], vj = s_vt[jl];
                    const real dx = pi.x + sx - pj.x, dy = pi.y + sy - pj.y, dz = pi.z + sz - pj.z;
                    const real r2 = dx * dx + dy * dy + dz * dz;
                    const real rinv = rsqrt_r(r2);
                    const real r = r2 * rinv;
                    const real w = (real)1 - r;
                    const real ex = dx * rinv, ey = dy * rinv, ez = dz * rinv;
                    const real evel = ex * (vi.x - vj.x) + ey * (vi.y - vj.y) + ez * (vi.z - vj.z);
                    const int tj = (int)pj.w;
                    const real aij = s_a[ti * nt + tj];
                    const int32_t idj = P::unpack_id(vj.w);
                    const uint32_t lo = (uint32_t)min(idi, idj), hi = (uint32_t)max(idi, idj);
                    const uint2 rnd = philox_xy(lo, hi, s_lo, s_hi, a.key0, a.key1);
                    const real th = theta_of(rnd, a.noise, (real)0);
                    const real fc = aij * w;
                    const real mag = fc - a.gamma * w * w * evel + a.sig_sqdt * w * th;
                    fx += mag * ex;
                    fy += mag * ey;
                    fz += mag * ez;
                    if (SAMPLE) {
                        wc += r * fc;
                        ep += (real)0.5 * fc * w;
                    }
                }
            }
        }
        if (active) {
            a.fpair[g] = mk4<vec4, real>(fx, fy, fz, (real)0);
            if (SAMPLE) a.ev[g] = mk4<vec4, real>(wc, ep, (real)0, (real)0);
        }
    }
}

// --------------------------------------------------------------------------
// a6-a7: bonded terms (eqs. 6-8, Fig. 3a) from a per-bead CSR table, the
// velocity update of Fig. 1 step 5, and the new force becomes f.
// --------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void bond_force(int kind, R r0, R k, R alpha, R dx, R dy, R dz, R &fx,
                                           R &fy, R &fz, R &U) {
    const R r2 = dx * dx + dy * dy + dz * dz;
    const R r = sqrt(r2);
    R coef = 0;
    U = 0;
    if (kind == 1) {
        if (r0 == (R)0) {
            coef = -k;
            U = (R)0.5 * k * r2;
        } else {
            U = (R)0.5 * k * (r - r0) * (r - r0);
            if (r > (R)0) coef = -k * (r - r0) / r;
        }
    } else if (kind == 2) {
        const R e = exp(-alpha * fabs(r - r0));
        U = k * ((R)1 - e) * ((R)1 - e);
        if (r > (R)0) coef = -(R)2 * k * alpha * e * ((R)1 - e) / r;
    } else if (kind == 3) {
        const R x = exp(-alpha * (r - r0));
        U = k * (((R)1 - x) * ((R)1 - x) - (R)1);
        if (r > (R)0) coef = -(R)2 * k * alpha * x * ((R)1 - x) / r;
    }
    fx = coef * dx;
    fy = coef * dy;
    fz = coef * dz;
}

template <class P>
struct BondArgs {
    using vec4 = typename P::vec4;
    using real = typename P::real;
    int n;
    Geo g;
    real L[3], h[3];
    real half_dt;
    const vec4 *fpair, *pos;
    const uint32_t *key;
    const int32_t *id, *inv_perm;
    const int32_t *bptr, *bpartner;
    const vec4 *bpar;      // r0, k, alpha, kind
    vec4 *vel, *frc, *ev;
};

template <class P>
__device__ __forceinline__ void bond_disp(const BondArgs<P> &a, int t, int u,
                                          typename P::real &dx, typename P::real &dy,
                                          typename P::real &dz) {
    using real = typename P::real;
    const typename P::vec4 pi = a.pos[t], pj = a.pos[u];
    if (P::kOffsets) {
        int xi, yi, zi, xj, yj, zj;
        decode_key(a.key[t], a.g, xi, yi, zi);
        decode_key(a.key[u], a.g, xj, yj, zj);
        int ddx = xi - xj, ddy = yi - yj, ddz = zi - zj;   // nearest periodic image in cells
        if (2 * ddx > a.g.nx) ddx -= a.g.nx; else if (2 * ddx < -a.g.nx) ddx += a.g.nx;
        if (2 * ddy > a.g.ny) ddy -= a.g.ny; else if (2 * ddy < -a.g.ny) ddy += a.g.ny;
        if (2 * ddz > a.g.nz) ddz -= a.g.nz; else if (2 * ddz < -a.g.nz) ddz += a.g.nz;
        dx = (pi.x - pj.x) + (real)ddx * a.h[0];
        dy = (pi.y - pj.y) + (real)ddy * a.h[1];
        dz = (pi.z - pj.z) + (real)ddz * a.h[2];
    } else {
        dx = pi.x - pj.x;
        dy = pi.y - pj.y;
        dz = pi.z - pj.z;
        dx -= a.L[0] * rint(dx / a.L[0]);
        dy -= a.L[1] * rint(dy / a.L[1]);
        dz -= a.L[2] * rint(dz / a.L[2]);
    }
}

template <class P, bool INIT, bool SAMPLE>
__global__ void __launch_bounds__(256) k_bond_vel(BondArgs<P> a) {
    using real = typename P::real;
    using vec4 = typename P::vec4;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n) return;
    const vec4 fp = a.fpair[t];
    real fx = fp.x, fy = fp.y, fz = fp.z, wb = 0, eb = 0;
    const int32_t i = a.id[t];
    const int b0 = a.bptr[i], b1 = a.bptr[i + 1];
    for (int b = b0; b < b1; ++b) {
        const int u = a.inv_perm[a.bpartner[b]];
        const vec4 bp = a.bpar[b];
        real dx, dy, dz, gx, gy, gz, U;
        bond_disp<P>(a, t, u, dx, dy, dz);
        bond_force<real>((int)bp.w, bp.x, bp.y, bp.z, dx, dy, dz, gx, gy, gz, U);
        fx += gx; fy += gy; fz += gz;
        if (SAMPLE) {
            wb += dx * gx + dy * gy + dz * gz;
            eb += U;
        }
    }
    if (!INIT) {
        const vec4 v = a.vel[t], f = a.frc[t];
        a.vel[t] = mk4<vec4, real>(v.x + a.half_dt * (f.x + fx), v.y + a.half_dt * (f.y + fy),
                                   v.z + a.half_dt * (f.z + fz), (real)0);
    }
    a.frc[t] = mk4<vec4, real>(fx, fy, fz, (real)0);
    if (SAMPLE) {
        const vec4 e = a.ev[t];
        a.ev[t] = mk4<vec4, real>(e.x, e.y, wb, eb);
    }
}

// --------------------------------------------------------------------------
// a8: FP64 reductions.  Pass 1: fixed grid, per-block partial sums of
// (px, py, pz, v^2, wc, ep, wb, eb).  Pass 2: one block adds the partials in
// block order (deterministic) and updates the running means.
// --------------------------------------------------------------------------
constexpr int RED_T = 256, RED_BLOCKS = 304, RED_K = 8;

template <class P>
__global__ void __launch_bounds__(RED_T) k_reduce(int n, const typename P::vec4 *vel,
                                                  const typename P::vec4 *ev, double *partial) {
    double s[RED_K] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int t = blockIdx.x * RED_T + threadIdx.x; t < n; t += gridDim.x * RED_T) {
        const typename P::vec4 v = vel[t], e = ev[t];
        const double vx = v.x, vy = v.y, vz = v.z;
        s[0] += vx; s[1] += vy; s[2] += vz;
        s[3] += vx * vx + vy * vy + vz * vz;
        s[4] += (double)e.x; s[5] += (double)e.y; s[6] += (double)e.z; s[7] += (double)e.w;
    }
    __shared__ double sh[RED_T / 32][RED_K];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < RED_K; ++k) {
        double x = s[k];
#pragma unroll
        for (int o = 16; o; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[wid][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < RED_K) {
        double x = 0;
        for (int w = 0; w < RED_T / 32; ++w) x += sh[w][threadIdx.x];
        partial[blockIdx.x * RED_K + threadIdx.x] = x;
    }
}

// obs[0..7]: px, py, pz, sum v^2, W_C, E_pair, W_B, E_bond (pair/bond sums
// halved: every pair / bond was visited from both ends).
// acc[0..2]: sum of kT, sum of p_total, number of samples.
static __global__ void k_reduce_final(int nblocks, const double *partial, double *obs, double *acc,
                               int accumulate, double inv_3n3, double inv_3V, int *status) {
    __shared__ double r[RED_K];
    if (threadIdx.x < RED_K) {
        double x = 0;
        for (int b = 0; b < nblocks; ++b) x += partial[b * RED_K + threadIdx.x];
        r[threadIdx.x] = threadIdx.x >= 4 ? 0.5 * x : x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bool ok = true;
        for (int k = 0; k < RED_K; ++k) {
            obs[k] = r[k];
            ok = ok && isfinite(r[k]);
        }
        if (!ok) atomicOr(status, ST_NONFINITE);
        if (accumulate) {
            acc[0] += r[3] * inv_3n3;
            acc[1] += (r[3] + r[4] + r[6]) * inv_3V;
            acc[2] += 1.0;
        }
    }
}

// --------------------------------------------------------------------------
// State read-back and the cell-division inspection.
// --------------------------------------------------------------------------
template <class P>
__global__ void __launch_bounds__(256) k_unpermute(int n, Geo g, const typename P::vec4 *pos,
                                                   const uint32_t *key,
                                                   const typename P::vec4 *vel,
                                                   const typename P::vec4 *frc, const int32_t *id,
                                                   double *opos, double *ovel, double *ofrc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int i = id[t];
    const typename P::vec4 p = pos[t], v = vel[t], f = frc[t];
    double x = p.x, y = p.y, z = p.z;
    if (P::kOffsets) {
        int cx, cy, cz;
        decode_key(key[t], g, cx, cy, cz);
        x = wrap_exact((double)cx * g.h[0] + x, g.L[0]);
        y = wrap_exact((double)cy * g.h[1] + y, g.L[1]);
        z = wrap_exact((double)cz * g.h[2] + z, g.L[2]);
    }
    opos[3 * i] = x; opos[3 * i + 1] = y; opos[3 * i + 2] = z;
    ovel[3 * i] = v.x; ovel[3 * i + 1] = v.y; ovel[3 * i + 2] = v.z;
    ofrc[3 * i] = f.x; ofrc[3 * i + 1] = f.y; ofrc[3 * i + 2] = f.z;
}

static __global__ void __launch_bounds__(256) k_cells_out(int n, const uint32_t *key, const int32_t *id,
                                                   uint32_t *key_by_id, int64_t *order) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int i = id[t];
    key_by_id[i] = key[t];
    order[t] = i;
}

// g(r): unique pairs (slot j > slot i) within (2K+1)^3 cells, FP64 distances.
template <class P>
__global__ void __launch_bounds__(256) k_gr(int n, Geo g, int Kx, int Ky, int Kz,
                                            const typename P::vec4 *pos, const uint32_t *key,
                                            const uint32_t *cell_start, double rmax, double dr,
                                            int nbins, unsigned long long *counts) {
    extern __shared__ unsigned long long s_cnt[];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) s_cnt[b] = 0ull;
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        int cx, cy, cz;
        decode_key(key[t], g, cx, cy, cz);
        const typename P::vec4 pi = pos[t];
        for (int dz = -Kz; dz <= Kz; ++dz)
            for (int dy = -Ky; dy <= Ky; ++dy)
                for (int dx = -Kx; dx <= Kx; ++dx) {
                    const int xx = (cx + dx + 8 * g.nx) % g.nx;
                    const int yy = (cy + dy + 8 * g.ny) % g.ny;
                    const int zz = (cz + dz + 8 * g.nz) % g.nz;
                    const uint32_t c = ((uint32_t)zz * g.ny + yy) * g.nx + xx;
                    const int b = (int)cell_start[c], e = (int)cell_start[c + 1];
                    for (int u = max(b, t + 1); u < e; ++u) {
                        const typename P::vec4 pj = pos[u];
                        double d[3];
                        if (P::kOffsets) {
                            d[0] = ((double)pi.x - (double)pj.x) + (double)(-dx) * g.h[0];
                            d[1] = ((double)pi.y - (double)pj.y) + (double)(-dy) * g.h[1];
                            d[2] = ((double)pi.z - (double)pj.z) + (double)(-dz) * g.h[2];
                        } else {
                            const double pa[3] = {(double)pi.x, (double)pi.y, (double)pi.z};
                            const double pb[3] = {(double)pj.x, (double)pj.y, (double)pj.z};
#pragma unroll
                            for (int k = 0; k < 3; ++k) {
                                const double dd = __dsub_rn(pa[k], pb[k]);
                                d[k] = __dsub_rn(dd, __dmul_rn(g.L[k], rint(__ddiv_rn(dd, g.L[k]))));
                            }
                        }
                        const double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]),
                                                                         __dmul_rn(d[1], d[1])),
                                                              __dmul_rn(d[2], d[2])));
                        if (r < rmax) {
                            const int bin = (int)floor(__ddiv_rn(r, dr));
                            if (bin < nbins) atomicAdd(&s_cnt[bin], 1ull);
                        }
                    }
                }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
        if (s_cnt[b]) atomicAdd(&counts[b], s_cnt[b]);
}

}  // namespace dpd
