// Device code of the DPD step loop (arxiv 1804.06205, Fig. 1) for sm_103a.
// Included by engine_f32.cu and engine_f64.cu (one precision each), by
// cells_noalloc.cu (cell keys and scans only) and by selfcheck.cu.
//
// Every kernel works on any number of resident systems at once: the systems
// are packed one after another in shared bead, cell, brick and bond pools, a
// per-system descriptor (SysDesc) holds geometry and parameters, and each
// bead (bsys) and pair-kernel brick (brick_sys) names its system.  Because
// the packing is contiguous in beads and cells alike, one global counting
// sort orders all systems at once.  Ids, cell keys and Philox counters are
// local to a system, so a system computes the same numbers alone or packed.
//
// One step (Fig. 1), all on the device; each kernel starts with
// griddep_wait, so the host may launch them back to back with programmatic
// dependent launch:
//   k_update      1.-2. r += dt v + dt^2/2 f, periodic wrap, new cell key,
//                 cell occupancy histogram (atomics on counts); usually done
//                 instead by the previous step's k_bond_vel (update_bead)
//   k_scan*       3.    exclusive scan of the counts -> cell_start
//   k_scatter     3.    slot = cell_start[key] + arrival rank
//   k_gather      3.    canonical (cell, id) order: each arrival ranks itself among
//                       its cell's ids and moves its state there; v~ = v + lambda dt f
//   k_pair        4.    eq. 3-4 + dissipative/random pair terms, 27-cell full shell
//   k_bond_vel    4.-5. eqs. 6-8 bonded terms, then v += dt/2 (f + f')
//   k_reduce*           FP64 sums for the observables (steps that sample running
//                       means; observables asked for between steps, after a
//                       sampled k_pair and k_bond_obs)
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
// Element w of a position holds the bead type and w of v~ the bead id, both
// as the bit pattern of the integer (pack_int), so no conversion is spent on
// them in the pair loop.
// --------------------------------------------------------------------------
struct __align__(32) dvec4 {
    double x, y, z, w;
};

struct PF32 {
    using real = float;
    using vec4 = float4;
    static constexpr bool kOffsets = true;
    static __device__ __forceinline__ real pack_int(int32_t i) { return __int_as_float(i); }
    static __device__ __forceinline__ int32_t unpack_int(real w) { return __float_as_int(w); }
};

struct PF64 {
    using real = double;
    using vec4 = dvec4;
    static constexpr bool kOffsets = false;
    static __device__ __forceinline__ real pack_int(int32_t i) {
        return __longlong_as_double((long long)i);
    }
    static __device__ __forceinline__ int32_t unpack_int(real w) {
        return (int32_t)__double_as_longlong(w);
    }
};

template <class V, class R>
__device__ __forceinline__ V mk4(R x, R y, R z, R w) {
    V v;
    v.x = x; v.y = y; v.z = z; v.w = w;
    return v;
}

// Programmatic dependent launch: wait until the preceding kernel in the
// stream has completed and its writes are visible (returns at once when the
// kernel was launched without the attribute).  The first statement of every
// kernel of a step.
__device__ __forceinline__ void griddep_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
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
    // ((x >> 8) | 1) * 2^-24 built without an int->float conversion: 1 + (x>>9)
    // 2^-23 by its bits, minus 1 - 2^-24 (exact: the operands are within a
    // factor 2 of each other, and the result (2 (x>>9) + 1) 2^-24 has 24 bits)
    return __fsub_rn(__uint_as_float(0x3F800000u | (x >> 9)), 0x1.fffffep-1f);
}
__device__ __forceinline__ double u01_f64(uint32_t x) {
    return (double)((x >> 8) | 1u) * 0x1p-24;
}

// Explicitly rounded arithmetic for the force terms: every kernel variant
// (sampled or not, initial or not) must produce the same bits, so the
// compiler may not fuse these differently from one variant to another.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
// the hardware's approximate reciprocal square root, base-2 logarithm and
// cosine with subnormal inputs flushed to zero: the same values as rsqrtf,
// __log2f and __cosf for every normal input and result
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_ftz(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float cos_ftz(float x) {
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }

// -2 ln(u) for the uniforms u = n 2^-24 (n odd, n < 2^24) of the FP64 path, by
// the table-driven method of P. T. P. Tang (ACM TOMS 16, 1990): with
// e = floor(log2 n) and j the next seven bits of n, n = 2^e (1 + j/128) + rest, and
//   ln u = (e - 24) ln 2 + ln(1 + j/128) + log1p(r),  r = rest 2^-e / (1 + j/128),
// |r| < 2^-7, log1p(r) by its Taylor series to r^7 / 7 (the next term is below
// 2e-18).  The reduction is integer arithmetic; the tables are filled with the
// library's log.  The tables and coefficients carry the factor -2 of Box-Muller:
// scaling by a power of two commutes with rounding, so every step, and the
// result, is exactly -2 times that of the same evaluation of ln u.  Ten FP64
// operations instead of a general log.
struct LnTab {
    double2 c[128];   // -2 ln(1 + j/128), 1 / (1 + j/128)
    double e[24];     // -2 (e - 24) ln 2
};
static __global__ void k_ln_tab(LnTab *t) {
    const int j = threadIdx.x;
    if (j < 128) {
        const double c = 1.0 + j / 128.0;
        t->c[j] = make_double2(-2.0 * log(c), 1.0 / c);
    }
    if (j < 24) t->e[j] = -2.0 * ((double)(j - 24) * log(2.0));
}
__device__ __forceinline__ double m2ln_u24(uint32_t n, const LnTab *t) {
    const int e = 31 - __clz(n);
    int j;
    uint32_t rest;
    if (e >= 7) {
        j = (int)((n >> (e - 7)) & 127u);
        rest = n & ((1u << (e - 7)) - 1u);
    } else {
        j = (int)((n << (7 - e)) & 127u);
        rest = 0u;
    }
    const double2 cj = t->c[j];
    // (1 + j/128)^-1 2^-e through the exponent field: exact, no underflow for e < 24
    const double inv = __longlong_as_double(__double_as_longlong(cj.y) - ((long long)e << 52));
    const double r = (double)rest * inv;
    double p = fma(r, -2.0 / 7.0, 2.0 / 6.0);
    p = fma(r, p, -2.0 / 5.0);
    p = fma(r, p, 2.0 / 4.0);
    p = fma(r, p, -2.0 / 3.0);
    p = fma(r, p, 2.0 / 2.0);
    p = fma(r, p, -2.0);
    return t->e[e] + fma(r, p, cj.x);
}
// cos(2 pi v) for the uniforms v = a 2^-24 (a odd, a < 2^24) of the FP64 path.
// The quadrant is a's top two bits, so the reduction is exact integer
// arithmetic: with b the remaining 22 bits, 2 pi v = q pi/2 + (pi/2) b 2^-22,
// and cos(q pi/2 + phi) = +-cos(psi) with psi = phi (q even) or pi/2 - phi (q
// odd), psi = (pi/2) c 2^-22 in [0, pi/2].  cos(psi) is its Taylor series to
// psi^20 / 20! (the next term is below 2e-17 in absolute value).
__device__ __forceinline__ double cos_u24(uint32_t a) {
    const uint32_t q = a >> 22, b = a & 0x3FFFFFu;
    const uint32_t c = (q & 1u) ? 0x400000u - b : b;
    const double psi = (double)c * (3.141592653589793 / 8388608.0);   // c pi 2^-23, pi/2^23 exact
    const double s = psi * psi;
    double p = 1.0 / 2432902008176640000.0;
    p = fma(s, p, -1.0 / 6402373705728000.0);
    p = fma(s, p, 1.0 / 20922789888000.0);
    p = fma(s, p, -1.0 / 87178291200.0);
    p = fma(s, p, 1.0 / 479001600.0);
    p = fma(s, p, -1.0 / 3628800.0);
    p = fma(s, p, 1.0 / 40320.0);
    p = fma(s, p, -1.0 / 720.0);
    p = fma(s, p, 1.0 / 24.0);
    p = fma(s, p, -1.0 / 2.0);
    p = fma(s, p, 1.0);
    return (q == 1u || q == 2u) ? -p : p;
}

// theta from Box-Muller on outputs 0 and 1 (noise 0) or sqrt(3)(2u-1) (noise 1).
__device__ __forceinline__ double theta_of(uint2 x, int noise, const LnTab *lt) {
    if (noise) return 1.7320508075688772 * (2.0 * u01_f64(x.x) - 1.0);
    return sqrt(m2ln_u24((x.x >> 8) | 1u, lt)) * cos_u24((x.y >> 8) | 1u);
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
// The same value as wrap_exact without a division, for x in [-L, 2L): there
// x/L rounds to a q in {-1, 0, 1, 2} whose x - L q is exact or x + L, and the
// two fix-ups map every such case onto x, x - L or x + L, as below.
__device__ __forceinline__ double wrap_fast(double x, double L) {
    if (!(x >= -L && x < 2.0 * L)) return wrap_exact(x, L);
    double y = x;
    if (y < 0.0) y = __dadd_rn(y, L);
    else if (y >= L) y = __dsub_rn(y, L);
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
// Per-system descriptor.
// --------------------------------------------------------------------------
template <class P>
struct SysDesc {
    using real = typename P::real;
    int n, bead0, cell0, ncell;      // beads [bead0, bead0+n), cells [cell0, cell0+ncell)
    int nx, ny, nz, ntypes;
    int brick0, X, BY, BZ;           // pair-kernel bricks [brick0, brick0 + nbx*nby*nbz)
    int nbx, nby, nbz, cap;          // cap: staged beads per brick chunk
    int a_off, noise, pad0, pad1;    // a_ij table offset, noise kind
    double L[3], h[3], inv_h[3];
    float hf[3], inv_hf[3];          // FP32 cell edges (offset path)
    real dt, half_dt2, half_dt, lam_dt, gamma, sig_sqdt;
    uint32_t rk[20];                 // Philox round keys
};

__device__ __forceinline__ void decode_key3(uint32_t k, int nx, int ny, int &cx, int &cy, int &cz) {
    cx = (int)(k % (uint32_t)nx);
    const uint32_t q = k / (uint32_t)nx;
    cy = (int)(q % (uint32_t)ny);
    cz = (int)(q / (uint32_t)ny);
}

// --------------------------------------------------------------------------
// a1-a2: position update, wrap, key (and set_state's initial binning).
// --------------------------------------------------------------------------
template <class P>
__device__ __forceinline__ void place_bead(const SysDesc<P> &D, double x, double y, double z,
                                           typename P::real type, typename P::vec4 &out,
                                           uint32_t &key, int *status, int bad_bit) {
    using real = typename P::real;
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) atomicOr(status, bad_bit);
    x = wrap_fast(x, D.L[0]);
    y = wrap_fast(y, D.L[1]);
    z = wrap_fast(z, D.L[2]);
    const int cx = cell_of(x, D.inv_h[0], D.nx);
    const int cy = cell_of(y, D.inv_h[1], D.ny);
    const int cz = cell_of(z, D.inv_h[2], D.nz);
    key = ((uint32_t)cz * (uint32_t)D.ny + (uint32_t)cy) * (uint32_t)D.nx + (uint32_t)cx;
    if (P::kOffsets) {
        out = mk4<typename P::vec4, real>((real)(x - (double)cx * D.h[0]),
                                          (real)(y - (double)cy * D.h[1]),
                                          (real)(z - (double)cz * D.h[2]), type);
    } else {
        out = mk4<typename P::vec4, real>((real)x, (real)y, (real)z, type);
    }
}

// FP32 path: the offset moves by the FP32 displacement and whole cells move
// to the integer cell index, wrapped periodically -- the absolute position is
// never formed.  FP64 path: x + displacement, wrapped in FP64.
__device__ __forceinline__ int move_cell(float &o, float h, float inv_h, int c, int n) {
    int d = (int)floorf(o * inv_h);
    o = fmaf(-(float)d, h, o);
    if (o < 0.0f) {
        o += h;
        --d;
    }
    if (o >= h) {
        o -= h;
        ++d;
    }
    int cc = (c + d) % n;
    return cc < 0 ? cc + n : cc;
}

// Fig. 1 steps 1-2 for one bead: r += dt v + dt^2/2 f, wrapped, and its new
// cell.  Shared by k_update and by the bond/velocity kernel, which does it for
// the next step while v and f are still in registers, so both give the same
// bits.
template <class P>
__device__ __forceinline__ void update_bead(const SysDesc<P> &D, const typename P::vec4 &p,
                                            uint32_t key_in, const typename P::vec4 &v,
                                            const typename P::vec4 &f, typename P::vec4 &out,
                                            uint32_t &key, int *status) {
    using real = typename P::real;
    const real dt = D.dt, hdt2 = D.half_dt2;
    const real ddx = fma_rn(hdt2, f.x, mul_rn(dt, v.x));
    const real ddy = fma_rn(hdt2, f.y, mul_rn(dt, v.y));
    const real ddz = fma_rn(hdt2, f.z, mul_rn(dt, v.z));
    if (P::kOffsets) {
        int cx, cy, cz;
        decode_key3(key_in, D.nx, D.ny, cx, cy, cz);
        float ox = add_rn((float)p.x, (float)ddx), oy = add_rn((float)p.y, (float)ddy),
              oz = add_rn((float)p.z, (float)ddz);
        if (!(isfinite(ox) && isfinite(oy) && isfinite(oz))) {
            atomicOr(status, ST_NONFINITE);
            ox = oy = oz = 0.0f;
        }
        cx = move_cell(ox, D.hf[0], D.inv_hf[0], cx, D.nx);
        cy = move_cell(oy, D.hf[1], D.inv_hf[1], cy, D.ny);
        cz = move_cell(oz, D.hf[2], D.inv_hf[2], cz, D.nz);
        key = ((uint32_t)cz * (uint32_t)D.ny + (uint32_t)cy) * (uint32_t)D.nx + (uint32_t)cx;
        out = mk4<typename P::vec4, real>((real)ox, (real)oy, (real)oz, p.w);
    } else {
        place_bead<P>(D, add_rn((double)p.x, (double)ddx), add_rn((double)p.y, (double)ddy),
                      add_rn((double)p.z, (double)ddz), p.w, out, key, status, ST_NONFINITE);
    }
}

template <class P>
struct UpdArgs {
    using vec4 = typename P::vec4;
    int b_lo, b_hi;
    const SysDesc<P> *sys;
    const int *bsys;
    int sys1;                        // the only system of a batch of one, else -1
    const uint32_t *key;             // local cell keys
    const vec4 *pos, *vel, *frc;
    vec4 *pos_tmp;
    uint32_t *key_tmp, *rank, *count;
    long long *counter;              // per system
    int *status;
};

// The system of bead t: a batch of one system needs no map.
template <class A>
__device__ __forceinline__ int bead_sys(const A &a, int t) {
    return a.sys1 >= 0 ? a.sys1 : a.bsys[t];
}

template <class P>
__device__ __forceinline__ void update_one(const UpdArgs<P> &a, int t) {
    const int s = bead_sys(a, t);
    const SysDesc<P> &D = a.sys[s];
    if (t == D.bead0) a.counter[s] += 1;   // evaluation counter of this step's force
    typename P::vec4 out;
    uint32_t key;
    update_bead<P>(D, a.pos[t], a.key[t], a.vel[t], a.frc[t], out, key, a.status);
    a.pos_tmp[t] = out;
    a.key_tmp[t] = key;
    a.rank[t] = atomicAdd(&a.count[D.cell0 + key], 1u);
}

template <class P>
__global__ void __launch_bounds__(256) k_update(UpdArgs<P> a) {
    griddep_wait();
    const int t = a.b_lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (t < a.b_hi) update_one<P>(a, t);
}

// set_state of one system: host positions/velocities in bead-id order
template <class P>
struct InitArgs {
    using vec4 = typename P::vec4;
    int s;
    const SysDesc<P> *sys;
    const double *pos_in, *vel_in;   // [n*3] bead-id order
    const int32_t *types;            // [n]
    vec4 *pos_tmp, *vel, *frc;       // at slots bead0 + id
    uint32_t *key_tmp, *rank, *count;
    int32_t *id;
    int *status;
    int i0, i1;                      // the bead ids [i0, i1) of this launch
};

template <class P>
__global__ void __launch_bounds__(256) k_init(InitArgs<P> a) {
    using real = typename P::real;
    const SysDesc<P> &D = a.sys[a.s];
    const int i = a.i0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.i1) return;
    const int t = D.bead0 + i;
    typename P::vec4 out;
    uint32_t key;
    place_bead<P>(D, a.pos_in[3 * i], a.pos_in[3 * i + 1], a.pos_in[3 * i + 2],
                  P::pack_int(a.types[i]), out, key, a.status, ST_BADINPUT);
    a.pos_tmp[t] = out;
    a.key_tmp[t] = key;
    a.rank[t] = atomicAdd(&a.count[D.cell0 + key], 1u);
    const double vx = a.vel_in[3 * i], vy = a.vel_in[3 * i + 1], vz = a.vel_in[3 * i + 2];
    if (!(isfinite(vx) && isfinite(vy) && isfinite(vz))) atomicOr(a.status, ST_BADINPUT);
    a.vel[t] = mk4<typename P::vec4, real>((real)vx, (real)vy, (real)vz, (real)0);
    a.frc[t] = mk4<typename P::vec4, real>((real)0, (real)0, (real)0, (real)0);
    a.id[t] = i;
}

// --------------------------------------------------------------------------
// a3: counting sort.  Exclusive scan of the per-cell counts: block sums
// (k_scan1), then block scans plus the sum of the preceding blocks
// (k_scan3b), which also clears the counts for the next step.  k_scan2 scans
// the block sums in one block for the allocation-free cell division.
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

// the SCAN_V counts of cells [b0, b0 + SCAN_V), zero past n: two 16-byte
// loads when the run is whole and aligned
__device__ __forceinline__ void load_counts(const uint32_t *count, int b0, int n,
                                            uint32_t (&v)[SCAN_V]) {
    static_assert(SCAN_V == 8, "two 16-byte loads");
    if (b0 + SCAN_V <= n && ((uintptr_t)(count + b0) & 15u) == 0) {
        const uint4 a = *reinterpret_cast<const uint4 *>(count + b0);
        const uint4 b = *reinterpret_cast<const uint4 *>(count + b0 + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int k = 0; k < SCAN_V; ++k) v[k] = (b0 + k < n) ? count[b0 + k] : 0u;
    }
}

// stores v[0..SCAN_V) at p[b0..) (only below n): two 16-byte stores when whole and aligned
__device__ __forceinline__ void store_run(uint32_t *p, int b0, int n, const uint32_t (&v)[SCAN_V]) {
    if (b0 + SCAN_V <= n && ((uintptr_t)(p + b0) & 15u) == 0) {
        *reinterpret_cast<uint4 *>(p + b0) = make_uint4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<uint4 *>(p + b0 + 4) = make_uint4(v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
        for (int k = 0; k < SCAN_V; ++k)
            if (b0 + k < n) p[b0 + k] = v[k];
    }
}

static __global__ void __launch_bounds__(SCAN_T) k_scan1(const uint32_t *count, int ncell,
                                                  uint32_t *bsum) {
    griddep_wait();
    const int base = blockIdx.x * SCAN_B + threadIdx.x * SCAN_V;
    uint32_t v[SCAN_V];
    load_counts(count, base, ncell, v);
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_V; ++k) s += v[k];
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


// Second pass of the two-pass scan: each block adds up the sums of the blocks
// before it (a few hundred values) instead of waiting for a separate scan of
// the block sums; cell starts are offset by `base`, and the last block writes
// the end of the range.  The counts are cleared for the next step.
static __global__ void __launch_bounds__(SCAN_T) k_scan3b(uint32_t *count, int ncell,
                                                   const uint32_t *bsum, uint32_t *cell_start,
                                                   uint32_t base) {
    griddep_wait();
    __shared__ uint32_t tot;
    uint32_t before = 0;
    for (int j = threadIdx.x; j < (int)blockIdx.x; j += SCAN_T) before += bsum[j];
    block_excl_scan(before, &tot);
    before = tot;
    const int b0 = blockIdx.x * SCAN_B + threadIdx.x * SCAN_V;
    uint32_t v[SCAN_V];
    load_counts(count, b0, ncell, v);
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_V; ++k) sum += v[k];
    uint32_t run = block_excl_scan(sum, &tot) + before + base;
    uint32_t st[SCAN_V];
#pragma unroll
    for (int k = 0; k < SCAN_V; ++k) {
        st[k] = run;
        run += v[k];
    }
    store_run(cell_start, b0, ncell, st);
    const uint32_t zero[SCAN_V] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    store_run(count, b0, ncell, zero);
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_T - 1) cell_start[ncell] = run;
}


template <class P>
struct ScatterArgs {
    int b_lo, b_hi;
    const SysDesc<P> *sys;
    const int *bsys;
    int sys1;                        // the only system of a batch of one, else -1
    const uint32_t *key_tmp, *rank, *cell_start;
    const int32_t *id_old;
    uint2 *srcid;                    // per arrival slot: (source slot, id)
};

template <class P>
__device__ __forceinline__ void scatter_one(const ScatterArgs<P> &a, int t) {
    const int s = bead_sys(a, t);
    const uint32_t slot = a.cell_start[a.sys[s].cell0 + a.key_tmp[t]] + a.rank[t];
    a.srcid[slot] = make_uint2((uint32_t)t, (uint32_t)a.id_old[t]);
}

template <class P>
__global__ void __launch_bounds__(256) k_scatter(ScatterArgs<P> a) {
    griddep_wait();
    const int t = a.b_lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (t < a.b_hi) scatter_one<P>(a, t);
}

template <class P>
struct GatherArgs {
    using vec4 = typename P::vec4;
    int b_lo, b_hi;
    const SysDesc<P> *sys;
    const int *bsys;
    int sys1;                        // the only system of a batch of one, else -1
    const uint2 *srcid;              // per arrival slot: (source slot, id)
    const uint32_t *cell_start;
    const vec4 *pos_tmp, *vel_old, *frc_old;
    const uint32_t *key_tmp;
    vec4 *pos, *vel, *frc, *vt;
    uint32_t *key;
    int32_t *id, *inv_perm;          // inv_perm: null when no system has bonds
    uint32_t *from;                  // source slot of every new slot (null: not kept)
};

// Atomic ranks put the beads of a cell in arrival order.  Each arrival finds
// its canonical place, the cell's start plus the number of the cell's beads
// with a smaller id (cells hold ~3 beads), and moves its state there.
// MOVE_VF: also move v and f into the new order (set_state and checkpoint
// restores); a step leaves them in the old order, where the bond/velocity
// kernel reads them through the source slot.
template <class P, bool MOVE_VF>
__device__ __forceinline__ void gather_one(const GatherArgs<P> &a, int t) {
    const SysDesc<P> &D = a.sys[bead_sys(a, t)];
    const uint2 si = a.srcid[t];
    const uint32_t s = si.x;
    const int32_t i = (int32_t)si.y;
    const uint32_t k = a.key_tmp[s];
    const uint32_t c = (uint32_t)D.cell0 + k;
    const int b = (int)a.cell_start[c], e = (int)a.cell_start[c + 1];
    int u = b;
    for (int q = b; q < e; ++q) u += (int32_t)a.srcid[q].y < i;
    const typename P::vec4 v = a.vel_old[s], f = a.frc_old[s];
    const typename P::real lam_dt = D.lam_dt;
    a.pos[u] = a.pos_tmp[s];
    a.key[u] = k;
    if (MOVE_VF) {
        a.vel[u] = v;
        a.frc[u] = f;
    }
    if (a.from) a.from[u] = s;
    a.id[u] = i;
    if (a.inv_perm) a.inv_perm[D.bead0 + i] = u;
    // Fig. 1 step 2: velocity predictor used by the dissipative force
    a.vt[u] = mk4<typename P::vec4, typename P::real>(v.x + lam_dt * f.x, v.y + lam_dt * f.y,
                                                      v.z + lam_dt * f.z, P::pack_int(i));
}

template <class P, bool MOVE_VF>
__global__ void __launch_bounds__(256) k_gather(GatherArgs<P> a) {
    griddep_wait();
    const int t = a.b_lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (t < a.b_hi) gather_one<P, MOVE_VF>(a, t);
}

// --------------------------------------------------------------------------
// a4-a5: pair forces, 27-cell full shell: every bead's force is summed in a
// fixed order by one thread, with no floating-point atomics.
//
// A block owns a brick of X x BY x BZ home cells (BY, BZ <= 2).  It stages the
// (BY+2)(BZ+2) neighbouring x-row runs (X+2 cells each, periodic) into shared
// memory with bulk copies, issued as soon as the runs' source ranges are
// known -- positions in the brick's frame (cell index relative to the
// brick, times h, plus the offset; FP64: the absolute position moved by the
// run's periodic image) and v~.  A home bead's 27 neighbour cells are 9 rows
// of 3 consecutive staged cells; a row, or its first or last cell, is skipped
// when its box lies at least r_c from the bead.
//
// Each warp takes 32 home beads (one per lane) and alternates two phases:
//   scan     every lane records its hits r^2 < 1 in row and slot order in its
//            own queue, at most PAIR_HMAX per pass (binary32 on both paths;
//            FP64 queues every pair with binary32 r^2 < 1.001 and the
//            evaluation applies the exact FP64 test);
//   evaluate every lane evaluates its own queue in order (FP32: two entries
//            per iteration, added in queue order) and adds the pair forces
//            to its bead's sums in registers.  FP64, when a block
//            needs one chunk and one pass: thread t evaluates the queue of
//            the block's bead of rank t by hit count, so that a warp's
//            queues have similar lengths (idle lanes still hold the FP64
//            pipe); when that pass holds every home bead, each pair of two
//            home beads is evaluated by one of them, which hands the other
//            its share as exact fixed point (integer atomics, so the sum
//            does not depend on their order).
// Passes repeat until all 27 cells are done; oversized neighbourhoods are
// staged in chunks.  Each bead's force is summed in a fixed order, so runs
// are deterministic; another brick shape changes only the order of the
// staged rows and so the rounding of the sums.
// --------------------------------------------------------------------------
template <class P>
struct PairArgs {   // one brick's system, as the kernel body uses it
    using vec4 = typename P::vec4;
    using real = typename P::real;
    const vec4 *pos, *vt;
    const uint32_t *key, *cell_start;   // cell_start offset to the system's cells
    vec4 *fpair, *ev;
    const real *a;                      // the system's a_ij table
    int ntypes;
    int nx, ny, nz;
    int X, BY, BZ, nbx, nby;
    real h[3];
    real gamma, sig_sqdt;
    int noise;
    const long long *counter;
    int cap;
};

template <class P>
struct PairLaunch {   // a launch over bricks [br_lo, br_lo + gridDim.x) of any systems
    using vec4 = typename P::vec4;
    using real = typename P::real;
    const SysDesc<P> *sys;
    const int *brick_sys;
    int sys1;                           // the only system of a batch of one, else -1
    int br_lo;
    int capmax, Xmax;                   // shared-memory layout
    const vec4 *pos, *vt;
    const uint32_t *key, *cell_start;
    vec4 *fpair, *ev;
    const real *atab;
    const long long *counter;
    int *status;                        // sticky status bits (ST_TIMEOUT)
    int ntmax;                          // largest number of bead types (a_ij table size)
    const LnTab *lntab;                 // FP64: tables of the Box-Muller logarithm
};

constexpr int PAIR_MAXX = 64;          // largest brick length (cells)
constexpr int PAIR_MAXT = 16;          // largest number of bead types
constexpr int PAIR_HMAX = 32;          // hits per lane per pass
constexpr int PAIR_NR = 16;            // staged rows, (2+2) x (2+2)
static_assert(PAIR_HMAX >= 1 && PAIR_HMAX <= 64, "hit queue length");
constexpr int PAIR_THREADS_PER_SM = 896; // FP32 register budget: 28 warps per SM
constexpr int PAIR64_THREADS_PER_SM = 384; // FP64 register budget: 12 warps per SM
constexpr int PAIR_PC = 3;             // ints per staged run: source, slot, length

template <class P>
struct PairSmem {
    static __host__ __device__ size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }
    static size_t bytes(int cap, int X, int T, int ntmax, bool sample) {
        using real = typename P::real;
        using vec4 = typename P::vec4;
        size_t b = 2 * (size_t)cap * sizeof(vec4);                 // staged positions, v~
        if (!P::kOffsets) b += (size_t)cap * sizeof(float4);      // FP64: their binary32 copies
        b += 2 * PAIR_NR * (size_t)(X + 3) * sizeof(int);          // staged cell starts; FP64 ranks
        b += PAIR_NR * 3 * PAIR_PC * sizeof(int) + 4 * 4 * sizeof(int);   // runs, home rows
        b += PAIR_NR * sizeof(int);                                // row keys
        b = align16(b);
        b += (size_t)ntmax * ntmax * sizeof(real) + PAIR_NR * 2 * sizeof(real);
        b = align16(b);
        const size_t nw = (size_t)T / 32;
        b += nw * PAIR_HMAX * 32 * sizeof(uint16_t);               // hit queues
        if (!P::kOffsets) {   // FP64 pairs of two home beads: partner shares, home index
            b = align16(b);
            b += 3 * (size_t)T * sizeof(unsigned long long);
            b += (size_t)cap * sizeof(int16_t);
        }
        (void)sample;
        return b;
    }
};

// Bulk asynchronous copies global -> shared (cp.async.bulk, completed on an
// mbarrier as a byte count) and the mbarrier operations they need.  Addresses
// and sizes must be multiples of 16 bytes.
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
// Shared-memory accesses by 32-bit shared-window address (the scan loop).
__device__ __forceinline__ float4 lds128(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(a));
    return v;
}
__device__ __forceinline__ void sts16(uint32_t a, uint32_t v) {
    asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t *m) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(m)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// orders this thread's earlier generic-proxy shared accesses before later
// async-proxy (bulk copy) accesses to the same memory
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *m, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *m) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                     smem_u32(m))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false if the phase has not completed after `tries` polls
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *m, uint32_t parity, int tries) {
    for (int i = 0; i < tries; ++i)
        if (mbar_try_wait(m, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *m) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(m))
        : "memory");
}
constexpr int MBAR_TRIES = 1 << 22;

// Philox4x32-10 with precomputed round keys (outputs 0 and 1).
__device__ __forceinline__ uint2 philox_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                           const uint32_t *rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk[2 * r];
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk[2 * r + 1];
        c0 = n0; c1 = (uint32_t)p1; c2 = n2; c3 = (uint32_t)p0;
    }
    return make_uint2(c0, c1);
}

// Box-Muller with the fast intrinsics (FP32 path): -2 ln u0 = -2 ln2 log2 u0,
// cos(2 pi u1) = -cos(2 pi u1 - pi) with the argument in (-pi, pi).
__device__ __forceinline__ float theta_pair(uint2 x, int noise, float, const LnTab *) {
    const float u0 = u01_f32(x.x);
    if (noise) return 1.7320508075688772f * (2.0f * u0 - 1.0f);
    const float u1 = u01_f32(x.y);
    const float q = fmaxf(-1.3862943611198906f * lg2_ftz(u0), 0.0f);
    const float s = q > 0.0f ? q * rsqrt_ftz(q) : 0.0f;
    return -s * cos_ftz(fmaf(6.2831853071795865f, u1, -3.1415926535897932f));
}
__device__ __forceinline__ double theta_pair(uint2 x, int noise, double, const LnTab *lt) {
    return theta_of(x, noise, lt);
}

// One block computes the pair forces of the home beads of one brick (T threads).
// Returns false (in every thread) if a staging copy never completed.  REUSE:
// the block goes on to another brick, so the staging mbarrier is invalidated
// at the end (it is initialised again at the start of the next brick).
template <class P, int T, bool SAMPLE, bool REUSE = false>
__device__ __forceinline__ bool pair_brick(const PairLaunch<P> &la, const int brick) {
    using real = typename P::real;
    using vec4 = typename P::vec4;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(32) unsigned char smem[];
    // this block's brick and system
    const int sysi = la.sys1 >= 0 ? la.sys1 : la.brick_sys[brick];
    const SysDesc<P> &D = la.sys[sysi];
    PairArgs<P> a;
    a.pos = la.pos;
    a.vt = la.vt;
    a.key = la.key;
    a.cell_start = la.cell_start + D.cell0;
    a.fpair = la.fpair;
    a.ev = la.ev;
    a.a = la.atab + D.a_off;
    a.ntypes = D.ntypes;
    a.nx = D.nx;
    a.ny = D.ny;
    a.nz = D.nz;
    a.X = D.X;
    a.BY = D.BY;
    a.BZ = D.BZ;
    a.nbx = D.nbx;
    a.nby = D.nby;
    a.h[0] = (real)D.h[0];
    a.h[1] = (real)D.h[1];
    a.h[2] = (real)D.h[2];
    a.gamma = D.gamma;
    a.sig_sqdt = D.sig_sqdt;
    uint32_t rkl[20];   // block-uniform round keys
#pragma unroll
    for (int r = 0; r < 20; ++r) rkl[r] = D.rk[r];
    a.noise = D.noise;
    a.counter = la.counter + sysi;
    a.cap = la.capmax;
    const int cap = la.capmax;
    const int X = a.X;
    vec4 *s_pos = reinterpret_cast<vec4 *>(smem);
    vec4 *s_vt = s_pos + cap;
    // FP64 path: binary32 copies of the staged frame positions, for the scan
    float4 *s_p32 = reinterpret_cast<float4 *>(s_vt + cap);
    int *s_cs = reinterpret_cast<int *>(s_p32 + (P::kOffsets ? 0 : cap));
    int *s_src = s_cs + PAIR_NR * (la.Xmax + 3);   // FP64: the balanced evaluation's ranks
    int *s_pc = s_src + PAIR_NR * (la.Xmax + 3);   // per source run: source slot, staged slot, length
    int *s_hr = s_pc + PAIR_NR * 3 * PAIR_PC;        // home rows: staged row, first, count, global
    int *s_rkey = s_hr + 16;                         // per staged row: key of its cell x = 0
    size_t off = PairSmem<P>::align16((size_t)((unsigned char *)(s_rkey + PAIR_NR) - smem));
    real *s_a = reinterpret_cast<real *>(smem + off);
    real *s_rsh = s_a + la.ntmax * la.ntmax;         // per staged row: y, z frame shift
    off = PairSmem<P>::align16((size_t)((unsigned char *)(s_rsh + 2 * PAIR_NR) - smem));
    uint16_t *s_q = reinterpret_cast<uint16_t *>(smem + off);   // per-lane hit queues
    // FP64: each home bead's share of the pairs that a home partner evaluated
    // (x, y, z; two's-complement fixed point in units of 2^-41), and the home
    // index of each staged slot (-1: not a home bead)
    off = PairSmem<P>::align16(off + (size_t)(T / 32) * PAIR_HMAX * 32 * sizeof(uint16_t));
    unsigned long long *s_acc = reinterpret_cast<unsigned long long *>(smem + off);
    int16_t *s_hidx = reinterpret_cast<int16_t *>(s_acc + 3 * T);

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    __shared__ __align__(8) uint64_t s_mbar;   // completion of the staging copies
    if (tid == 0) {
        mbar_init(&s_mbar, 1);
        fence_mbar_init();
    }
    uint32_t mphase = 0;
    int bid = brick - D.brick0;
    const int bx = bid % a.nbx;
    bid /= a.nbx;
    const int byi = bid % a.nby, bzi = bid / a.nby;
    const int x0 = bx * X, y0 = byi * a.BY, z0 = bzi * a.BZ;
    const int Xe = min(X, a.nx - x0), BYe = min(a.BY, a.ny - y0), BZe = min(a.BZ, a.nz - z0);
    const int W = Xe + 3;                 // staged cells per row (ux = -1..Xe) + row end
    const int SY = BYe + 2, NRe = SY * (BZe + 2);
    const real hx = a.h[0], hy = a.h[1], hz = a.h[2];

    for (int e = tid; e < a.ntypes * a.ntypes; e += T) s_a[e] = a.a[e];
    // The (row, cell) grid of the neighbourhood is shared by all threads; a
    // thread's position in it advances by T without any division.
    const int gr0 = tid / W, gk0 = tid - gr0 * W, gdr = T / W, gdk = T - gdr * W;
    // A staged row of X + 2 cells (k = 0..Xe+1 <-> ux = -1..Xe) is at most three
    // contiguous source runs, split where x wraps: at k = 1 when x0 = 0, and
    // where x0 + k - 1 = nx.  Run j covers cells [kb_j, kb_{j+1}), kb_0 = 0;
    // -1: no such run.
    const int kw = a.nx - x0 + 1;
    const bool w1 = x0 == 0, w2 = kw <= Xe + 1;
    const int kend = Xe + 2;
    const int kb1 = w1 ? 1 : (w2 ? kw : kend);
    const int kb2 = w1 ? (w2 ? kw : kend) : (w2 ? kend : -1);
    const int kb3 = (w1 && w2) ? kend : -1;
    auto run_of = [&](int k) { return k >= kb1 ? ((kb2 >= 0 && k >= kb2) ? 2 : 1) : 0; };
    auto wrap_x = [&](int k) {   // the periodic x of staged cell k
        const int xx = x0 + k - 1;
        return xx + (xx < 0 ? a.nx : (xx >= a.nx ? -a.nx : 0));
    };
    auto row_key = [&](int r) {   // key of the (wrapped) staged row's cell x = 0
        const int uy = r % SY - 1, uz = r / SY - 1;
        int yy = y0 + uy, zz = z0 + uz;
        yy += yy < 0 ? a.ny : (yy >= a.ny ? -a.ny : 0);
        zz += zz < 0 ? a.nz : (zz >= a.nz ? -a.nz : 0);
        return ((uint32_t)zz * a.ny + yy) * a.nx;
    };
    if (tid < NRe) {   // each staged row's first key and frame shift
        const int r = tid;
        const int uy = r % SY - 1, uz = r / SY - 1;
        int yy = y0 + uy, zz = z0 + uz;
        yy += yy < 0 ? a.ny : (yy >= a.ny ? -a.ny : 0);
        zz += zz < 0 ? a.nz : (zz >= a.nz ? -a.nz : 0);
        s_rkey[r] = (int)(((uint32_t)zz * a.ny + yy) * a.nx);
        real sy, sz;
        if (P::kOffsets) {       // offset -> brick frame
            sy = mul_rn((real)uy, hy);
            sz = mul_rn((real)uz, hz);
        } else {                 // absolute -> brick frame, undoing the row's wrap
            sy = mul_rn((real)(uy - yy), hy);
            sz = mul_rn((real)(uz - zz), hz);
        }
        s_rsh[2 * r] = sy;
        s_rsh[2 * r + 1] = sz;
    }
    if (tid < NRe * 3) {   // run j of row r: its source range, from two cell starts
        const int r = tid / 3, j = tid - 3 * r;
        const int k0 = j == 0 ? 0 : (j == 1 ? kb1 : kb2);
        const int k1 = j == 0 ? kb1 : (j == 1 ? kb2 : kb3);
        int src = 0, len = 0;
        if (k1 > k0) {
            const uint32_t rk = row_key(r);
            src = (int)a.cell_start[rk + (uint32_t)wrap_x(k0)];
            len = (int)a.cell_start[rk + (uint32_t)wrap_x(k1 - 1) + 1u] - src;
        }
        s_pc[tid * PAIR_PC] = src;        // first source slot
        s_pc[tid * PAIR_PC + 2] = len;    // length
    }
    __syncthreads();
    __shared__ int s_total;
    if (tid < 32) {   // first staged slot of each run: exclusive scan over the runs in order
        const int n3 = NRe * 3;   // at most 48
        const int v0 = tid < n3 ? s_pc[tid * PAIR_PC + 2] : 0;
        const int v1 = tid + 32 < n3 ? s_pc[(tid + 32) * PAIR_PC + 2] : 0;
        int i0 = v0, i1 = v1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u0 = __shfl_up_sync(FULL, i0, o), u1 = __shfl_up_sync(FULL, i1, o);
            if (tid >= o) {
                i0 += u0;
                i1 += u1;
            }
        }
        const int t0 = __shfl_sync(FULL, i0, 31);
        if (tid < n3) s_pc[tid * PAIR_PC + 1] = i0 - v0;
        if (tid + 32 < n3) s_pc[(tid + 32) * PAIR_PC + 1] = t0 + i1 - v1;
        if (tid == 31) s_total = t0 + i1;
    }
    __syncthreads();
    const int S = s_total;
    const int c1_first = min(S, cap);
    // Staging of slots [c0, c1) of the neighbourhood, in two parts.  issue: bulk
    // copies of each source run (positions, v~) onto the mbarrier.  complete:
    // wait for them, then move every staged cell into the brick's frame.  False
    // if a copy never completed (the block must then leave).
    auto issue = [&](int c0, int c1) {
        fence_proxy_async_smem();   // this chunk's reads before the next copies
        __syncthreads();            // everyone is done with the previous chunk
        if (tid < NRe * 3) {        // one thread per source run: positions, v~
            const int *pc = s_pc + tid * PAIR_PC;
            const int src = pc[0], dst = pc[1], len = pc[2];
            const int lo = max(dst, c0), hi = min(dst + len, c1);
            if (lo < hi) {
                const uint32_t bytes = (uint32_t)(hi - lo) * (uint32_t)sizeof(vec4);
                mbar_expect_tx(&s_mbar, 2u * bytes);
                bulk_g2s(s_pos + (lo - c0), a.pos + src + (lo - dst), bytes, &s_mbar);
                bulk_g2s(s_vt + (lo - c0), a.vt + src + (lo - dst), bytes, &s_mbar);
            }
        }
    };
    auto complete = [&](int c0, int c1) -> bool {
        __syncthreads();            // every copy issued before the arrival
        if (tid == 0) mbar_arrive(&s_mbar);
        const bool got = mbar_wait_bounded(&s_mbar, mphase, MBAR_TRIES);
        mphase ^= 1u;
        if (__syncthreads_or(!got)) {   // a copy never completed: flag it, leave
            if (tid == 0) atomicOr(la.status, ST_TIMEOUT);
            mbar_wait_bounded(&s_mbar, mphase ^ 1u, MBAR_TRIES);
            return false;
        }
        // into the brick's frame, cell by cell: x by the cell's place in
        // the brick, y and z by the row's shift
        int r = gr0 - gdr, k = gk0 - gdk;
        for (int e = tid; e < NRe * W; e += T) {
            k += gdk;
            r += gdr;
            if (k >= W) {
                k -= W;
                ++r;
            }
            if (k > Xe + 1) continue;                 // the row-end entry
            const int lo = max(s_cs[e], c0), hi = min(s_cs[e + 1], c1);
            if (lo >= hi) continue;
            real sx;
            if (P::kOffsets) {
                sx = (real)(k - 1);
            } else {   // absolute x -> brick frame, undoing the cell's wrap
                int cx = x0 + k - 1;
                cx += cx < 0 ? a.nx : (cx >= a.nx ? -a.nx : 0);
                sx = mul_rn((real)(k - 1 - cx), hx);
            }
            const real sy = s_rsh[2 * r], sz = s_rsh[2 * r + 1];
            for (int q = lo; q < hi; ++q) {
                vec4 p = s_pos[q - c0];
                if (P::kOffsets) p.x = fma_rn(sx, hx, p.x);
                else p.x = add_rn(p.x, sx);
                p.y = add_rn(p.y, sy);
                p.z = add_rn(p.z, sz);
                s_pos[q - c0] = p;
                if (!P::kOffsets)
                    s_p32[q - c0] = make_float4((float)p.x, (float)p.y, (float)p.z, 0.0f);
            }
        }
        __syncthreads();   // staged and moved before anyone scans
        return true;
    };
    // The first chunk's copies are in flight while the staged start of every
    // cell (k = Xe+2: the row end) is formed from its run's staged start and
    // its own cell start.
    issue(0, c1_first);
    bool first_pending = true;
    {
        int r = gr0, k = gk0;
#pragma unroll 2
        for (int e = tid; e < NRe * W; e += T) {
            int st;
            if (k <= Xe + 1) {
                const int *pc = s_pc + (r * 3 + run_of(k)) * PAIR_PC;
                st = pc[1] + (int)a.cell_start[(uint32_t)s_rkey[r] + (uint32_t)wrap_x(k)] - pc[0];
            } else {
                const int *pe = s_pc + (r * 3 + 2) * PAIR_PC;
                st = pe[1] + pe[2];
            }
            s_cs[e] = st;
            k += gdk;
            r += gdr;
            if (k >= W) {
                k -= W;
                ++r;
            }
        }
    }
    __syncthreads();
    if (tid < 4) {     // home rows (ry, rz) = (tid % 2, tid / 2)
        const int ry = tid % 2, rz = tid / 2;
        int hcount = 0, first = 0, gfirst = 0, sr = 0;
        if (ry < BYe && rz < BZe) {
            sr = (ry + 1) + SY * (rz + 1);
            const int *pc = s_pc + (sr * 3 + run_of(1)) * PAIR_PC;
            gfirst = pc[0] + s_cs[sr * W + 1] - pc[1];    // global slot of cell k = 1's first bead
            hcount = s_cs[sr * W + Xe + 1] - s_cs[sr * W + 1];
        }
        s_hr[4 * tid] = sr;
        s_hr[4 * tid + 1] = first;
        s_hr[4 * tid + 2] = hcount;
        s_hr[4 * tid + 3] = gfirst;
    }
    __syncthreads();
    if (tid == 0) {    // home rows' positions in the concatenated home list
        int run = 0;
        for (int h = 0; h < 4; ++h) {
            s_hr[4 * h + 1] = run;
            run += s_hr[4 * h + 2];
        }
    }
    __syncthreads();
    const int H = s_hr[13] + s_hr[14];
    const long long sctr = *a.counter;
    const uint32_t s_lo = (uint32_t)(unsigned long long)sctr;
    const uint32_t s_hi = (uint32_t)((unsigned long long)sctr >> 32);
    const int nt = a.ntypes;
    uint16_t *my_q = s_q + wid * PAIR_HMAX * 32;
    auto stage = [&](int c0, int c1) -> bool {
        issue(c0, c1);
        return complete(c0, c1);
    };
    int staged_lo = -1;
    // FP64: balanced evaluation (ranks in s_src, which holds PAIR_NR * (Xmax + 3) ints)
    const bool balance = !P::kOffsets && PAIR_NR * (la.Xmax + 3) >= T;

    for (int hb0 = 0; hb0 < H; hb0 += T) {
        const int hb = hb0 + tid;
        const bool active = hb < H;
        // which home row, global slot, frame coordinates
        int hr = 0;
        if (active)
            while (hr < 3 && hb >= s_hr[4 * (hr + 1) + 1]) ++hr;
        const int g = active ? s_hr[4 * hr + 3] + (hb - s_hr[4 * hr + 1]) : 0;
        const int ry = hr % 2, rz = hr / 2;
        const int sr_home = s_hr[4 * hr];
        // this bead's state from global memory; the loads are in flight while
        // the first chunk is staged
        const vec4 pr = a.pos[g], hv = a.vt[g];
        const uint32_t kg = a.key[g];
        if (staged_lo != 0) {
            if (first_pending) {
                if (!complete(0, c1_first)) return false;
                first_pending = false;
            } else if (!stage(0, c1_first)) {
                return false;
            }
            staged_lo = 0;
        }
        int uxi = 0;
        vec4 hp = pr;
        if (active) {
            const uint32_t rowkey = ((uint32_t)(z0 + rz) * a.ny + (y0 + ry)) * a.nx;
            uxi = (int)(kg - rowkey) - x0;
            // the same operations as the staging of this bead's own copy, so the
            // two coincide bit for bit and the self pair has r^2 == 0 exactly
            if (P::kOffsets) {
                hp.x = fma_rn((real)uxi, hx, pr.x);
                hp.y = add_rn(pr.y, mul_rn((real)ry, hy));
                hp.z = add_rn(pr.z, mul_rn((real)rz, hz));
            } else {
                hp.x = add_rn(pr.x, mul_rn((real)(-x0), hx));
                hp.y = add_rn(pr.y, mul_rn((real)(-y0), hy));
                hp.z = add_rn(pr.z, mul_rn((real)(-z0), hz));
            }
        }
        real ax = 0, ay = 0, az = 0, aw = 0, ae = 0;   // this bead's sums
        // distances from the bead to the faces of its cell (pruning); the scan
        // runs in binary32 on both paths (FP64: on binary32 copies of the
        // positions, with margins far above their rounding)
        const float lxd = (float)(hp.x - (real)uxi * hx), uxd = (float)hx - lxd;
        const float lyd = (float)(hp.y - (real)ry * hy), uyd = (float)hy - lyd;
        const float lzd = (float)(hp.z - (real)rz * hz), uzd = (float)hz - lzd;
        const float cut2 = 1.0001f;
        // FP32: a hit is 2^-126 <= r^2 < 1 (the bead's staged copy coincides with it);
        // FP64: r^2 < 1.001 in binary32 and not the bead itself, and the exact
        // test is made in the evaluation, so the hits summed are the same
        constexpr float scan_lim = P::kOffsets ? 1.0f : 1.001f;
        const float4 *s_scan = P::kOffsets ? reinterpret_cast<const float4 *>(s_pos) : s_p32;
        const int self_abs = active ? s_cs[sr_home * W + 1] + (hb - s_hr[4 * hr + 1]) : -1;

        // FP64, one pass over every home bead: each pair of two home beads is
        // evaluated by one of them (once), which sets wide if a share did not fit
        bool once = false, wide = false;
        // the queue qb[m * 32 + col], m < n, of the bead at ip (v~ iv): each
        // lane takes its entries in scan order and adds them to the sums
        auto evaluate = [&](const uint16_t *qb, int col, int n, const vec4 &ip, const vec4 &iv,
                            real &sx, real &sy, real &sz, real &sw, real &se) {
                const int nmax = (int)__reduce_max_sync(FULL, (unsigned)n);
                if constexpr (P::kOffsets) {
                    // binary32: pj - pi and vj - vi (negated differences, the same r^2
                    // and e.v) with x and y packed; each term is added to the sums with
                    // one explicit fused multiply-add (x and y packed, kept negated),
                    // so every kernel variant rounds the sums the same way
                    const float2 nip = make_float2(-ip.x, -ip.y), niv = make_float2(-iv.x, -iv.y);
                    float2 ns = make_float2(0.0f - sx, 0.0f - sy);
                    // one queue entry: the pair's magnitude and the unit vector from
                    // i to j (x, y packed), and the sampled terms
                    auto term = [&](int jl, float &mag, float2 &e, float &ez, float &rr1,
                                    float &fc, float &w) {
                        const vec4 pj = s_pos[jl], vj = s_vt[jl];
                        const float2 d = __fadd2_rn(make_float2(pj.x, pj.y), nip);
                        const float dzv = pj.z - ip.z;
                        const float r2 = fma_rn(dzv, dzv, fma_rn(d.y, d.y, mul_rn(d.x, d.x)));
                        const float rinv = rsqrt_ftz(r2);
                        rr1 = mul_rn(r2, rinv);
                        w = 1.0f - rr1;
                        e = __fmul2_rn(d, make_float2(rinv, rinv));
                        ez = mul_rn(dzv, rinv);
                        const float2 dv = __fadd2_rn(make_float2(vj.x, vj.y), niv);
                        const float evel = fma_rn(ez, vj.z - iv.z, fma_rn(e.y, dv.y, mul_rn(e.x, dv.x)));
                        const float aij = s_a[P::unpack_int(ip.w) * nt + P::unpack_int(pj.w)];
                        const int32_t idi = P::unpack_int(iv.w), idj = P::unpack_int(vj.w);
                        const uint32_t lo = (uint32_t)min(idi, idj), hi = (uint32_t)max(idi, idj);
                        const uint2 rnd = philox_rk(lo, hi, s_lo, s_hi, rkl);
                        const float th = theta_pair(rnd, a.noise, 0.0f, la.lntab);
                        fc = mul_rn(aij, w);
                        const float gw2 = mul_rn(mul_rn(a.gamma, w), w);
                        mag = fma_rn(mul_rn(a.sig_sqdt, w), th, fma_rn(-gw2, evel, fc));
                    };
                    // two entries per iteration, independent until they are added in order
                    for (int m = 0; m < nmax; m += 2) {
                        if (m < n) {
                            const bool two = m + 1 < n;
                            const int j0 = qb[m * 32 + col];
                            const int j1 = two ? (int)qb[(m + 1) * 32 + col] : j0;
                            float mag0, ez0, rr0, fc0, w0, mag1, ez1, rr1_, fc1, w1;
                            float2 e0, e1;
                            term(j0, mag0, e0, ez0, rr0, fc0, w0);
                            term(j1, mag1, e1, ez1, rr1_, fc1, w1);
                            ns = __ffma2_rn(make_float2(mag0, mag0), e0, ns);
                            sz = __fmaf_rn(-mag0, ez0, sz);
                            if (SAMPLE) {
                                sw += rr0 * fc0;
                                se += 0.5f * fc0 * w0;
                            }
                            if (two) {
                                ns = __ffma2_rn(make_float2(mag1, mag1), e1, ns);
                                sz = __fmaf_rn(-mag1, ez1, sz);
                                if (SAMPLE) {
                                    sw += rr1_ * fc1;
                                    se += 0.5f * fc1 * w1;
                                }
                            }
                        }
                    }
                    sx = 0.0f - ns.x;
                    sy = 0.0f - ns.y;
                } else {   // FP64
                    for (int m = 0; m < nmax; ++m) {
                        if (m < n) {
                            const int jl = qb[m * 32 + col];
                            const vec4 pj = s_pos[jl], vj = s_vt[jl];
                            const real dx = ip.x - pj.x, dyv = ip.y - pj.y, dzv = ip.z - pj.z;
                            const real r2 = fma_rn(dzv, dzv, fma_rn(dyv, dyv, mul_rn(dx, dx)));
                            if (!P::kOffsets && !(r2 < (real)1 && r2 > (real)0)) continue;
                            const real rinv = rsqrt_r(r2);
                            const real rr1 = mul_rn(r2, rinv);
                            const real w = (real)1 - rr1;
                            // e.v_ij = (d.v_ij) / r; F = w S e with S = a_ij - gamma w e.v_ij
                            // + sigma theta / sqrt(dt), added as (w / r) S d, w / r = 1/r - 1
                            const real dvx = iv.x - vj.x, dvy = iv.y - vj.y, dvz = iv.z - vj.z;
                            const real evel = mul_rn(fma_rn(dzv, dvz, fma_rn(dyv, dvy, mul_rn(dx, dvx))), rinv);
                            const real aij = s_a[P::unpack_int(ip.w) * nt + P::unpack_int(pj.w)];
                            const int32_t idi = P::unpack_int(iv.w), idj = P::unpack_int(vj.w);
                            const uint32_t lo = (uint32_t)min(idi, idj), hi = (uint32_t)max(idi, idj);
                            const uint2 rnd = philox_rk(lo, hi, s_lo, s_hi, rkl);
                            const real th = theta_pair(rnd, a.noise, (real)0, la.lntab);
                            const real S = fma_rn(a.sig_sqdt, th, fma_rn(-mul_rn(a.gamma, w), evel, aij));
                            const real magr = mul_rn(rinv - (real)1, S);
                            sx = fma_rn(magr, dx, sx);
                            sy = fma_rn(magr, dyv, sy);
                            sz = fma_rn(magr, dzv, sz);
                            bool both = false;   // this pair's terms count for both beads
                            if (once) {
                                const int hj = s_hidx[jl];
                                if (hj >= 0) {
                                    // a home partner: it receives -F in fixed point (units of
                                    // 2^-41, exact sums in any order).  With |F_c| <= |magr| r
                                    // < 2^9 (from the exponents of magr and r) a share is
                                    // below 2^50, so one fused multiply-add with 1.5 * 2^52
                                    // rounds it to an integer held in the low bits, and the
                                    // sum of at most PAIR_HMAX shares stays below 2^55
                                    both = true;
                                    const int em = (__double2hiint(magr) >> 20) & 0x7ff;
                                    const int er = (__double2hiint(rr1) >> 20) & 0x7ff;
                                    if (em + er <= 2 * 1023 + 7) {
                                        unsigned long long *acc = s_acc + 3 * hj;
                                        const real ms = mul_rn(magr, 0x1p41);
                                        const long long m52 = 0x4338000000000000ll;   // 1.5 * 2^52
                                        atomicAdd(acc, (unsigned long long)(m52 - __double_as_longlong(fma_rn(ms, dx, 0x1.8p52))));
                                        atomicAdd(acc + 1, (unsigned long long)(m52 - __double_as_longlong(fma_rn(ms, dyv, 0x1.8p52))));
                                        atomicAdd(acc + 2, (unsigned long long)(m52 - __double_as_longlong(fma_rn(ms, dzv, 0x1.8p52))));
                                    } else {
                                        wide = true;   // a large or non-finite force
                                    }
                                }
                            }
                            if (SAMPLE) {
                                const real fc = mul_rn(aij, w);
                                const real tw = rr1 * fc, te = (real)0.5 * fc * w;
                                sw += both ? tw + tw : tw;
                                se += both ? te + te : te;
                            }
                        }
                    }
                }
        };
        bool done = false;   // the forces were written by the balanced evaluation

        for (int c0 = 0; c0 < S; c0 += cap) {
            const int c1 = min(S, c0 + cap);
            if (staged_lo != c0) {
                if (!stage(c0, c1)) return false;
                staged_lo = c0;
            }
            __syncwarp();
            // minus the bead's coordinates: the scan forms pj - pi (the negated
            // difference, same r^2), x and y in one packed binary32 add
            const float2 nxy = make_float2(-(float)hp.x, -(float)hp.y);
            const float nzs = -(float)hp.z;
            const uint32_t self =
                (self_abs >= c0 && self_abs < c1) ? (uint32_t)(self_abs - c0) : 0xFFFFu;
            const uint32_t scan_u32 = smem_u32(s_scan), myq_u32 = smem_u32(my_q + lane);
            int r9 = 0, q = 0;
            bool more = active;
            // ---- scan: up to PAIR_HMAX hits, rows (dz, dy) ascending, slots ascending
            auto scan = [&](int &nh) {
                if (more) {
                    // the 9 rows unrolled (row offsets and face distances known at
                    // compile time); a pass resumes at row r9
                    bool stopped = false;
#pragma unroll(P::kOffsets ? 9 : 1)
                    for (int rr = 0; rr < 9; ++rr) {
                        if (rr < r9) continue;
                        r9 = rr;
                        const int dy = rr % 3 - 1, dz = rr / 3 - 1;
                        const float ey = dy < 0 ? lyd : (dy > 0 ? uyd : 0.0f);
                        const float ez = dz < 0 ? lzd : (dz > 0 ? uzd : 0.0f);
                        const float dyz = ey * ey + ez * ez;
                        if (dyz >= cut2) continue;                       // row out of reach
                        const int sr = sr_home + dy + SY * dz;
                        const int* cs = s_cs + sr * W + uxi;
                        const int qb = max(dyz + lxd * lxd < cut2 ? cs[0] : cs[1], c0);
                        const int qe_full = min(dyz + uxd * uxd < cut2 ? cs[3] : cs[2], c1);
                        if (q < qb) q = qb;
                        if (q >= qe_full) continue;
                        int qe = qe_full;
                        if (qe - q > PAIR_HMAX - nh) {
                            if (nh > 0) {                        // evaluate first, resume here
                                stopped = true;
                                break;
                            }
                            qe = q + PAIR_HMAX;                  // a crowded row: part of it
                        }
                        {   // queue [level][lane]: the staged slot of each hit, stored
                            // at the lane's next free level (a row never holds more
                            // candidates than free levels, so the stores stay in the
                            // queue).  Shared addresses are 32-bit window offsets; the
                            // next pair of candidates is loaded before this pair is
                            // tested
                            {
                            uint32_t ad = scan_u32 + 16u * (uint32_t)(q - c0);
                            const uint32_t ad_end = scan_u32 + 16u * (uint32_t)(qe - c0);
                            uint32_t ent = (uint32_t)(q - c0);
                            uint32_t qa = myq_u32 + 64u * (uint32_t)nh;
                            // one candidate: its hit is 2^-126 <= r^2 < 1 (FP32: the bits
                            // of a non-negative binary32 order like its value, so this is
                            // one unsigned compare of the bits minus those of 2^-126; a
                            // subnormal r^2, r < 1.1e-19, counts as coincident, like r = 0)
                            // or binary32 r^2 < 1.001 and not the bead itself (FP64)
                            auto hit = [&](const float4 &c, uint32_t e) -> bool {
                                const float2 d = __fadd2_rn(make_float2(c.x, c.y), nxy);
                                const float dzv = add_rn(c.z, nzs);
                                const float r2 = fma_rn(dzv, dzv, fma_rn(d.y, d.y, mul_rn(d.x, d.x)));
                                return P::kOffsets ? (__float_as_uint(r2) - 0x00800000u < 0x3F000000u)
                                                   : (r2 < scan_lim && e != self);
                            };
                            auto put = [&](bool h, uint32_t e) {
                                if (h) {
                                    sts16(qa, e);
                                    qa += 64u;
                                }
                            };
                            // two at a time, the next two loaded into the same registers
                            // once the tests have read them
                            float4 pa = lds128(ad), pb = lds128(ad + 16u);
                            while (ad + 16u < ad_end) {
                                const bool ha = hit(pa, ent), hb = hit(pb, ent + 1u);
                                ad += 32u;
                                pa = lds128(ad);
                                pb = lds128(ad + 16u);
                                put(ha, ent);
                                put(hb, ent + 1u);
                                ent += 2u;
                            }
                            if (ad < ad_end) { put(hit(pa, ent), ent); ++ent; }
                            q = (int)ent + c0;
                            nh = (int)((qa - myq_u32) >> 6);
                            }
                        }
                        if (q < qe_full) {
                            stopped = true;
                            break;
                        }
                    }
                    if (!stopped) r9 = 9;
                    more = r9 < 9;
                }
            };
            if (balance && S <= cap) {
                // FP64, one chunk: the first pass of every lane in the block, then,
                // if no lane needs another, thread t evaluates the queue of the bead
                // of rank t by hit count (most first), so that a warp's queues have
                // similar lengths: lanes left idle by short queues still occupy the
                // FP64 pipe.  Each bead's terms are added in scan order as before.
                // When the pass holds every home bead, each pair of two home beads
                // is evaluated once, by one of them, and the other one's queue drops
                // it: the FP64 pipe then computes about a third fewer pair terms.
                once = H <= T;
                for (;;) {
                    if (tid <= PAIR_HMAX) s_pc[tid] = 0;     // histogram of hit counts
                    int nh = 0;
                    scan(nh);
                    __syncwarp();
                    if (__syncthreads_or(more)) {
                        // some lane needs another pass: evaluate this one, then go on as usual
                        once = false;
                        evaluate(my_q, lane, nh, hp, hv, ax, ay, az, aw, ae);
                        __syncwarp();
                        break;
                    }
                    if (once) {
                        // the pair of home beads b, b' is evaluated by the lower index
                        // when b + b' is even, else by the higher, so that each bead
                        // keeps about half of its home pairs; shares start at zero
                        for (int e = tid; e < S; e += T) s_hidx[e] = -1;
                        s_acc[3 * tid] = s_acc[3 * tid + 1] = s_acc[3 * tid + 2] = 0ull;
                        __syncthreads();
                        if (active) s_hidx[self_abs] = (int16_t)hb;
                        __syncthreads();
                        if (active) {   // drop the pairs the partner evaluates, keep the order
                            int k = 0;
                            for (int m = 0; m < nh; ++m) {
                                const int e = my_q[m * 32 + lane];
                                const int hj = s_hidx[e];
                                if (hj < 0 || (((hb + hj) & 1) ? hb > hj : hb < hj))
                                    my_q[(k++) * 32 + lane] = (uint16_t)e;
                            }
                            nh = k;
                        }
                    }
                    if (active) atomicAdd(&s_pc[PAIR_HMAX - nh], 1);
                    __syncthreads();
                    if (tid < 32) {   // bin starts, most hits first
                        const int v = s_pc[tid];
                        int inc = v;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const int u = __shfl_up_sync(FULL, inc, o);
                            if (tid >= o) inc += u;
                        }
                        s_pc[tid] = inc - v;
                        if (tid == 31) s_pc[32] = inc;
                    }
                    __syncthreads();
                    if (active) s_src[atomicAdd(&s_pc[PAIR_HMAX - nh], 1)] = tid | (nh << 8);
                    __syncthreads();
                    const int nact = min(T, H - hb0);
                    int own = 0, on = 0, go = 0;
                    vec4 ip = hp, iv = hv;
                    if (tid < nact) {   // the bead of rank tid: its staged copy is its state
                        const int v = s_src[tid];
                        own = v & 255;
                        on = v >> 8;
                        const int ob = hb0 + own;
                        int orow = 0;
                        while (orow < 3 && ob >= s_hr[4 * (orow + 1) + 1]) ++orow;
                        const int k = ob - s_hr[4 * orow + 1];
                        go = s_hr[4 * orow + 3] + k;
                        const int oself = s_cs[s_hr[4 * orow] * W + 1] + k;
                        ip = s_pos[oself];
                        iv = s_vt[oself];
                    }
                    real bx = 0, by = 0, bz = 0, bw = 0, be = 0;
                    evaluate(s_q + (own >> 5) * PAIR_HMAX * 32, own & 31, on, ip, iv, bx, by, bz,
                             bw, be);
                    __syncwarp();
                    if (once) {
                        if (__syncthreads_or(wide)) {
                            // a share too large for the fixed point: the brick again,
                            // every pair from both ends (the scan restarts)
                            once = false;
                            r9 = 0;
                            q = 0;
                            more = active;
                            continue;
                        }
                        if (tid < nact) {   // the bead's own sum, then its partners' shares
                            const unsigned long long *acc = s_acc + 3 * own;
                            bx = add_rn(bx, mul_rn((real)(long long)acc[0], (real)0x1p-41));
                            by = add_rn(by, mul_rn((real)(long long)acc[1], (real)0x1p-41));
                            bz = add_rn(bz, mul_rn((real)(long long)acc[2], (real)0x1p-41));
                        }
                    }
                    if (tid < nact) {
                        a.fpair[go] = mk4<vec4, real>(bx, by, bz, (real)0);
                        if (SAMPLE) a.ev[go] = mk4<vec4, real>(bw, be, (real)0, (real)0);
                    }
                    done = true;
                    __syncthreads();   // every queue read before the next scan
                    break;
                }
                if (done) break;
            }
            while (__any_sync(FULL, more)) {
                int nh = 0;
                scan(nh);
                __syncwarp();
                evaluate(my_q, lane, nh, hp, hv, ax, ay, az, aw, ae);
                __syncwarp();
            }
        }
        if (active && !done) {
            a.fpair[g] = mk4<vec4, real>(ax, ay, az, (real)0);
            if (SAMPLE) a.ev[g] = mk4<vec4, real>(aw, ae, (real)0, (real)0);
        }
        __syncwarp();
    }
    // no home bead: the first chunk's copies must still land before the block
    // leaves or reuses its shared memory
    if (first_pending && !complete(0, c1_first)) return false;
    if (REUSE) {
        __syncthreads();
        if (tid == 0) mbar_inval(&s_mbar);
    }
    return true;
}

template <class P, int T, bool SAMPLE>
__global__ void __launch_bounds__(T, P::kOffsets ? PAIR_THREADS_PER_SM / T : (T <= PAIR64_THREADS_PER_SM ? PAIR64_THREADS_PER_SM / T : 1)) k_pair(PairLaunch<P> la) {
    griddep_wait();
    pair_brick<P, T, SAMPLE>(la, la.br_lo + blockIdx.x);
}

// --------------------------------------------------------------------------
// a6-a7: bonded terms (eqs. 6-8, Fig. 3a) from a per-bead CSR table, the
// velocity update of Fig. 1 step 5, and the new force becomes f.
// --------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void bond_force(int kind, R r0, R k, R alpha, R dx, R dy, R dz, R &fx,
                                           R &fy, R &fz, R &U) {
    // explicit rounding throughout: every kernel that calls this gets the same bits
    const R r2 = fma_rn(dz, dz, fma_rn(dy, dy, mul_rn(dx, dx)));
    const R r = sqrt(r2);
    R coef = 0;
    U = 0;
    if (kind == 1) {
        if (r0 == (R)0) {
            coef = -k;
            U = mul_rn(mul_rn((R)0.5, k), r2);
        } else {
            const R d = r - r0;
            U = mul_rn(mul_rn((R)0.5, k), mul_rn(d, d));
            if (r > (R)0) coef = mul_rn(-k, d) / r;
        }
    } else if (kind == 2) {
        const R e = exp(mul_rn(-alpha, fabs(r - r0)));
        const R om = (R)1 - e;
        U = mul_rn(mul_rn(k, om), om);
        if (r > (R)0) coef = mul_rn(mul_rn(mul_rn((R)-2 * k, alpha), e), om) / r;
    } else if (kind == 3) {
        const R x = exp(mul_rn(-alpha, r - r0));
        const R om = (R)1 - x;
        U = mul_rn(k, mul_rn(om, om) - (R)1);
        if (r > (R)0) coef = mul_rn(mul_rn(mul_rn((R)-2 * k, alpha), x), om) / r;
    }
    fx = mul_rn(coef, dx);
    fy = mul_rn(coef, dy);
    fz = mul_rn(coef, dz);
}

template <class P>
struct BondArgs {
    using vec4 = typename P::vec4;
    int b_lo, b_hi;
    const SysDesc<P> *sys;
    const int *bsys;
    int sys1;                        // the only system of a batch of one, else -1
    const vec4 *fpair, *pos;
    const uint32_t *key;
    const int32_t *id, *inv_perm;
    const int32_t *bptr;   // [bead0 + id] -> first record (pool offset)
    const int32_t *bpartner;   // partner's local id
    const vec4 *bpar;      // r0, k, alpha, kind
    // v and f of the step in the previous order, read through the source slot
    // of each bead (the sort's gather does not move them; it records the
    // source slots in `from`); written in the new order to vel, frc
    const uint32_t *from;
    const vec4 *vel_old, *frc_old;
    vec4 *vel, *frc, *ev;
    // the next step's update (FUSE): as UpdArgs
    vec4 *pos_tmp;
    uint32_t *key_tmp, *rank, *count;
    long long *counter;
    int *status;
};

template <class P>
__device__ __forceinline__ void bond_disp(const BondArgs<P> &a, const SysDesc<P> &D, int t, int u,
                                          typename P::real &dx, typename P::real &dy,
                                          typename P::real &dz) {
    using real = typename P::real;
    const typename P::vec4 pi = a.pos[t], pj = a.pos[u];
    if (P::kOffsets) {
        int xi, yi, zi, xj, yj, zj;
        decode_key3(a.key[t], D.nx, D.ny, xi, yi, zi);
        decode_key3(a.key[u], D.nx, D.ny, xj, yj, zj);
        int ddx = xi - xj, ddy = yi - yj, ddz = zi - zj;   // nearest periodic image in cells
        if (2 * ddx > D.nx) ddx -= D.nx; else if (2 * ddx < -D.nx) ddx += D.nx;
        if (2 * ddy > D.ny) ddy -= D.ny; else if (2 * ddy < -D.ny) ddy += D.ny;
        if (2 * ddz > D.nz) ddz -= D.nz; else if (2 * ddz < -D.nz) ddz += D.nz;
        dx = (pi.x - pj.x) + (real)ddx * (real)D.h[0];
        dy = (pi.y - pj.y) + (real)ddy * (real)D.h[1];
        dz = (pi.z - pj.z) + (real)ddz * (real)D.h[2];
    } else {
        dx = pi.x - pj.x;
        dy = pi.y - pj.y;
        dz = pi.z - pj.z;
        dx -= (real)D.L[0] * rint(dx / (real)D.L[0]);
        dy -= (real)D.L[1] * rint(dy / (real)D.L[1]);
        dz -= (real)D.L[2] * rint(dz / (real)D.L[2]);
    }
}

template <class P, bool INIT, bool SAMPLE, bool FUSE>
__device__ __forceinline__ void bond_vel_one(const BondArgs<P> &a, int t) {
    static_assert(!FUSE || !INIT, "the fused update follows a velocity update");
    using real = typename P::real;
    using vec4 = typename P::vec4;
    const int sysi = bead_sys(a, t);
    const SysDesc<P> &D = a.sys[sysi];
    const vec4 fp = a.fpair[t];
    real fx = fp.x, fy = fp.y, fz = fp.z, wb = 0, eb = 0;
    int b0 = 0, b1 = 0;
    if (a.bptr) {   // null when no resident system has bonds
        const int32_t i = a.id[t];
        b0 = a.bptr[D.bead0 + i];
        b1 = a.bptr[D.bead0 + i + 1];
    }
    for (int b = b0; b < b1; ++b) {
        const int u = a.inv_perm[D.bead0 + a.bpartner[b]];
        const vec4 bp = a.bpar[b];
        real dx, dy, dz, gx, gy, gz, U;
        bond_disp<P>(a, D, t, u, dx, dy, dz);
        bond_force<real>((int)bp.w, bp.x, bp.y, bp.z, dx, dy, dz, gx, gy, gz, U);
        fx = add_rn(fx, gx);
        fy = add_rn(fy, gy);
        fz = add_rn(fz, gz);
        if (SAMPLE) {   // rounded as in k_bond_obs, so both give the same bits
            wb = add_rn(wb, fma_rn(dz, gz, fma_rn(dy, gy, mul_rn(dx, gx))));
            eb = add_rn(eb, U);
        }
    }
    vec4 vn = mk4<vec4, real>((real)0, (real)0, (real)0, (real)0);
    const uint32_t so = a.from[t];
    if (!INIT) {
        const real hdt = D.half_dt;
        const vec4 v = a.vel_old[so], f = a.frc_old[so];
        vn = mk4<vec4, real>(v.x + hdt * (f.x + fx), v.y + hdt * (f.y + fy),
                             v.z + hdt * (f.z + fz), (real)0);
        a.vel[t] = vn;
    } else {   // the initial force: v stays, moved into the new order
        const vec4 v = a.vel_old[so];
        a.vel[t] = mk4<vec4, real>(v.x, v.y, v.z, (real)0);
    }
    const vec4 fn = mk4<vec4, real>(fx, fy, fz, (real)0);
    // the pair kernel writes into this force buffer itself (fpair == frc):
    // only a bead with bond terms changes it
    if (a.frc != a.fpair || b1 > b0) a.frc[t] = fn;
    if (!FUSE) {   // (the fused update checks the positions it makes)
        if (!isfinite(fx + fy + fz + vn.x + vn.y + vn.z)) atomicOr(a.status, ST_NONFINITE);
    }
    if (FUSE) {   // Fig. 1 steps 1-2 of the next step, from this step's v and f
        if (t == D.bead0) a.counter[sysi] += 1;
        vec4 out;
        uint32_t key;
        update_bead<P>(D, a.pos[t], a.key[t], vn, fn, out, key, a.status);
        a.pos_tmp[t] = out;
        a.key_tmp[t] = key;
        a.rank[t] = atomicAdd(&a.count[D.cell0 + key], 1u);
    }
    if (SAMPLE) {
        const vec4 e = a.ev[t];
        a.ev[t] = mk4<vec4, real>(e.x, e.y, wb, eb);
    }
}

template <class P, bool INIT, bool SAMPLE, bool FUSE = false>
__global__ void __launch_bounds__(256) k_bond_vel(BondArgs<P> a) {
    griddep_wait();
    const int t = a.b_lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (t < a.b_hi) bond_vel_one<P, INIT, SAMPLE, FUSE>(a, t);
}

// Bond virial and energy of every bead's bond records (ev.z, ev.w), from the
// current positions and nothing else written: the bond half of an observables
// pass made on demand, with the rounded accumulation of the sampled k_bond_vel.
template <class P>
__global__ void __launch_bounds__(256) k_bond_obs(BondArgs<P> a) {
    griddep_wait();
    using real = typename P::real;
    using vec4 = typename P::vec4;
    const int t = a.b_lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.b_hi) return;
    const SysDesc<P> &D = a.sys[bead_sys(a, t)];
    real wb = 0, eb = 0;
    int b0 = 0, b1 = 0;
    if (a.bptr) {
        const int32_t i = a.id[t];
        b0 = a.bptr[D.bead0 + i];
        b1 = a.bptr[D.bead0 + i + 1];
    }
    for (int b = b0; b < b1; ++b) {
        const int u = a.inv_perm[D.bead0 + a.bpartner[b]];
        const vec4 bp = a.bpar[b];
        real dx, dy, dz, gx, gy, gz, U;
        bond_disp<P>(a, D, t, u, dx, dy, dz);
        bond_force<real>((int)bp.w, bp.x, bp.y, bp.z, dx, dy, dz, gx, gy, gz, U);
        wb = add_rn(wb, fma_rn(dz, gz, fma_rn(dy, gy, mul_rn(dx, gx))));
        eb = add_rn(eb, U);
    }
    const vec4 e = a.ev[t];
    a.ev[t] = mk4<vec4, real>(e.x, e.y, wb, eb);
}

// --------------------------------------------------------------------------
// a8: FP64 reductions, per system.  Pass 1: each block adds one chunk of one
// system's beads, (px, py, pz, v^2, wc, ep, wb, eb).  Pass 2: one block per
// system adds its chunks in order (deterministic) and updates its running
// means.
// --------------------------------------------------------------------------
constexpr int RED_T = 256, RED_CHUNK = 4096, RED_K = 8;

// rmap[block] = (first bead slot, end slot); rsys[k] = (system, first block, blocks)
template <class P>
__global__ void __launch_bounds__(RED_T) k_reduce(const int2 *rmap, const typename P::vec4 *vel,
                                                  const typename P::vec4 *ev, double *partial) {
    griddep_wait();
    const int2 r = rmap[blockIdx.x];
    double s[RED_K] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int t = r.x + threadIdx.x; t < r.y; t += RED_T) {
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

// obs[s*8 + 0..7]: px, py, pz, sum v^2, W_C, E_pair, W_B, E_bond (pair/bond
// sums halved: every pair / bond was visited from both ends).
// acc[s*4 + 0..2]: sum of kT, sum of p_total, number of samples.
template <class P>
__global__ void __launch_bounds__(RED_T)
    k_reduce_final(const int4 *rsys, const SysDesc<P> *sys, const double *partial, double *obs,
                   double *acc, int accumulate, int *status) {
    griddep_wait();
    const int4 q = rsys[blockIdx.x];
    const int s = q.x;
    // every thread sums a strided share of the system's block partials, then
    // the block combines them (fixed order: the result does not depend on timing)
    double x[RED_K] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = q.y + (int)threadIdx.x; b < q.y + q.z; b += RED_T)
#pragma unroll
        for (int k = 0; k < RED_K; ++k) x[k] += partial[b * RED_K + k];
    __shared__ double sh[RED_T / 32][RED_K];
    __shared__ double r[RED_K];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < RED_K; ++k) {
        double v = x[k];
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < RED_K) {
        double v = 0;
        for (int w = 0; w < RED_T / 32; ++w) v += sh[w][threadIdx.x];
        r[threadIdx.x] = threadIdx.x >= 4 ? 0.5 * v : v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bool ok = true;
        for (int k = 0; k < RED_K; ++k) {
            obs[s * RED_K + k] = r[k];
            ok = ok && isfinite(r[k]);
        }
        if (!ok) atomicOr(status, ST_NONFINITE);
        if (accumulate) {
            const SysDesc<P> &D = sys[s];
            const double V = D.L[0] * D.L[1] * D.L[2];
            const double inv_3n3 = D.n > 1 ? 1.0 / (3.0 * D.n - 3.0) : 0.0;
            acc[4 * s] += r[3] * inv_3n3;
            acc[4 * s + 1] += (r[3] + r[4] + r[6]) / (3.0 * V);
            acc[4 * s + 2] += 1.0;
        }
    }
}

// --------------------------------------------------------------------------
// State read-back and the cell-division inspection (one system).
// --------------------------------------------------------------------------
// id -> slot map of one system's beads, for the gathering read-out below
static __global__ void __launch_bounds__(256) k_inv_perm(int bead0, int n, const int32_t *id,
                                                         int32_t *inv_perm) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    inv_perm[bead0 + id[bead0 + k]] = bead0 + k;
}

// One system's state in bead-id order, as doubles, for the ids [i0, i1):
// thread i gathers bead i from its slot (so the writes are contiguous), with
// absolute positions.
template <class P>
__global__ void __launch_bounds__(256) k_unpermute(int s, int i0, int i1, const SysDesc<P> *sys,
                                                   const typename P::vec4 *pos,
                                                   const uint32_t *key,
                                                   const typename P::vec4 *vel,
                                                   const typename P::vec4 *frc,
                                                   const int32_t *inv_perm,
                                                   double *opos, double *ovel, double *ofrc) {
    const SysDesc<P> &D = sys[s];
    const int i = i0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= i1) return;
    const int t = inv_perm[D.bead0 + i];
    const typename P::vec4 p = pos[t], v = vel[t], f = frc[t];
    double x = p.x, y = p.y, z = p.z;
    if (P::kOffsets) {
        int cx, cy, cz;
        decode_key3(key[t], D.nx, D.ny, cx, cy, cz);
        x = wrap_fast((double)cx * D.h[0] + x, D.L[0]);
        y = wrap_fast((double)cy * D.h[1] + y, D.L[1]);
        z = wrap_fast((double)cz * D.h[2] + z, D.L[2]);
    }
    opos[3 * i] = x; opos[3 * i + 1] = y; opos[3 * i + 2] = z;
    ovel[3 * i] = v.x; ovel[3 * i + 1] = v.y; ovel[3 * i + 2] = v.z;
    ofrc[3 * i] = f.x; ofrc[3 * i + 1] = f.y; ofrc[3 * i + 2] = f.z;
}

// --------------------------------------------------------------------------
// Checkpoints: the exact state (position representation, v, f) of one system
// in bead-id order, so that a restored system continues bit for bit.
// FP32 record: key, offset[3], v[3], f[3] (40 B); FP64: x[3], v[3], f[3] (72 B).
// --------------------------------------------------------------------------
struct CkptRec32 {
    uint32_t key;
    float o[3], v[3], f[3];
};
struct CkptRec64 {
    double x[3], v[3], f[3];
};
template <class P>
struct CkptRec;
template <>
struct CkptRec<PF32> {
    using type = CkptRec32;
};
template <>
struct CkptRec<PF64> {
    using type = CkptRec64;
};

// The records of a block (256 ids) move between the record array and shared
// memory as 8-byte words, so a warp's accesses are contiguous: the array may be
// host memory that the kernel reads or writes directly over the host link.
// The array must be 8-byte aligned (records are multiples of 8 bytes).
constexpr int CKPT_BLOCK = 256;

template <class P>
__global__ void __launch_bounds__(CKPT_BLOCK) k_ckpt_out(int s, int i0, int i1, const SysDesc<P> *sys,
                                                         const typename P::vec4 *pos, const uint32_t *key,
                                                         const typename P::vec4 *vel,
                                                         const typename P::vec4 *frc,
                                                         const int32_t *inv_perm,
                                                         typename CkptRec<P>::type *out) {
    using Rec = typename CkptRec<P>::type;
    constexpr int W = (int)(sizeof(Rec) / 8);
    static_assert(sizeof(Rec) % 8 == 0, "records are whole 8-byte words");
    __shared__ __align__(16) uint2 s_w[CKPT_BLOCK * W];
    const SysDesc<P> &D = sys[s];
    const int b0 = i0 + blockIdx.x * CKPT_BLOCK;   // ids [b0, b0 + cnt) of [i0, i1)
    const int cnt = min(CKPT_BLOCK, i1 - b0);
    const int i = b0 + threadIdx.x;
    if (i < i1) {
        const int t = inv_perm[D.bead0 + i];
        const typename P::vec4 p = pos[t], v = vel[t], f = frc[t];
        Rec r;
        if constexpr (P::kOffsets) {
            r.key = key[t];
            r.o[0] = p.x; r.o[1] = p.y; r.o[2] = p.z;
        } else {
            r.x[0] = p.x; r.x[1] = p.y; r.x[2] = p.z;
        }
        r.v[0] = v.x; r.v[1] = v.y; r.v[2] = v.z;
        r.f[0] = f.x; r.f[1] = f.y; r.f[2] = f.z;
        reinterpret_cast<Rec *>(s_w)[threadIdx.x] = r;
    }
    __syncthreads();
    uint2 *dst = reinterpret_cast<uint2 *>(out + b0);
    if ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {   // 16-byte words, an 8-byte tail
        const int n16 = cnt * W / 2;
        for (int k = threadIdx.x; k < n16; k += CKPT_BLOCK)
            reinterpret_cast<uint4 *>(dst)[k] = reinterpret_cast<const uint4 *>(s_w)[k];
        if (((cnt * W) & 1) && threadIdx.x == 0) dst[2 * n16] = s_w[2 * n16];
    } else {
        for (int k = threadIdx.x; k < cnt * W; k += CKPT_BLOCK) dst[k] = s_w[k];
    }
}

// Restore: like the initial binning (k_init), from checkpoint records; a
// non-finite value or an FP32 key beyond the system's cells sets ST_BADINPUT.
template <class P>
__global__ void __launch_bounds__(CKPT_BLOCK) k_ckpt_in(InitArgs<P> a,
                                                        const typename CkptRec<P>::type *rec) {
    using real = typename P::real;
    using Rec = typename CkptRec<P>::type;
    constexpr int W = (int)(sizeof(Rec) / 8);
    __shared__ uint2 s_w[CKPT_BLOCK * W];
    const SysDesc<P> &D = a.sys[a.s];
    const int b0 = a.i0 + blockIdx.x * CKPT_BLOCK;   // ids [b0, b0 + cnt) of [i0, i1)
    const int cnt = min(CKPT_BLOCK, a.i1 - b0);
    const uint2 *src = reinterpret_cast<const uint2 *>(rec + b0);
    for (int k = threadIdx.x; k < cnt * W; k += CKPT_BLOCK) s_w[k] = src[k];
    __syncthreads();
    const int i = b0 + threadIdx.x;
    if (i >= a.i1) return;
    const int t = D.bead0 + i;
    const Rec r = reinterpret_cast<const Rec *>(s_w)[threadIdx.x];
    typename P::vec4 out;
    uint32_t key;
    bool fin = isfinite(r.v[0]) && isfinite(r.v[1]) && isfinite(r.v[2]) && isfinite(r.f[0]) &&
               isfinite(r.f[1]) && isfinite(r.f[2]);
    if constexpr (P::kOffsets) {
        fin = fin && isfinite(r.o[0]) && isfinite(r.o[1]) && isfinite(r.o[2]);
        key = r.key;
        if (key >= (uint32_t)D.ncell) {   // refused by the host after the sync; clamped so
            fin = false;                  // that nothing reads or counts out of range
            key = 0u;
        }
        out = mk4<typename P::vec4, real>(r.o[0], r.o[1], r.o[2], P::pack_int(a.types[i]));
    } else {
        place_bead<P>(D, r.x[0], r.x[1], r.x[2], P::pack_int(a.types[i]), out, key, a.status,
                      ST_BADINPUT);
    }
    if (!fin) atomicOr(a.status, ST_BADINPUT);
    a.pos_tmp[t] = out;
    a.key_tmp[t] = key;
    if (a.count) a.rank[t] = atomicAdd(&a.count[D.cell0 + key], 1u);   // null: no sort follows
    a.vel[t] = mk4<typename P::vec4, real>(r.v[0], r.v[1], r.v[2], (real)0);
    a.frc[t] = mk4<typename P::vec4, real>(r.f[0], r.f[1], r.f[2], (real)0);
    a.id[t] = i;
}

// The state of beads [bead0, bead0 + n) of system s, held in any order, as the
// input of a cell division: position and key into the sort's work arrays with
// an arrival rank, v, f and id into the other ping-pong buffers.
template <class P>
__global__ void __launch_bounds__(256) k_resort_prep(int s, const SysDesc<P> *sys,
                                                     const typename P::vec4 *pos,
                                                     const uint32_t *key,
                                                     const typename P::vec4 *vel,
                                                     const typename P::vec4 *frc,
                                                     const int32_t *id,
                                                     typename P::vec4 *pos_tmp, uint32_t *key_tmp,
                                                     uint32_t *rank, uint32_t *count,
                                                     typename P::vec4 *vel_old,
                                                     typename P::vec4 *frc_old, int32_t *id_old) {
    const SysDesc<P> &D = sys[s];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= D.n) return;
    const int t = D.bead0 + k;
    const uint32_t c = key[t];
    pos_tmp[t] = pos[t];
    key_tmp[t] = c;
    rank[t] = atomicAdd(&count[D.cell0 + c], 1u);
    vel_old[t] = vel[t];
    frc_old[t] = frc[t];
    id_old[t] = id[t];
}

template <class P>
__global__ void __launch_bounds__(256) k_cells_out(int s, const SysDesc<P> *sys,
                                                   const uint32_t *key, const int32_t *id,
                                                   uint32_t *key_by_id, int64_t *order) {
    const SysDesc<P> &D = sys[s];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= D.n) return;
    const int i = id[D.bead0 + k];
    key_by_id[i] = key[D.bead0 + k];
    order[k] = i;
}

// g(r): unique pairs (slot j > slot i) within (2K+1)^3 cells, FP64 distances.
template <class P>
__global__ void __launch_bounds__(256) k_gr(int s, const SysDesc<P> *sys, int Kx, int Ky, int Kz,
                                            const typename P::vec4 *pos, const uint32_t *key,
                                            const uint32_t *cell_start, double rmax, double dr,
                                            int nbins, unsigned long long *counts) {
    extern __shared__ unsigned long long s_cnt[];
    const SysDesc<P> &D = sys[s];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) s_cnt[b] = 0ull;
    __syncthreads();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < D.n) {
        const int t = D.bead0 + k;
        int cx, cy, cz;
        decode_key3(key[t], D.nx, D.ny, cx, cy, cz);
        const typename P::vec4 pi = pos[t];
        for (int dz = -Kz; dz <= Kz; ++dz)
            for (int dy = -Ky; dy <= Ky; ++dy)
                for (int dx = -Kx; dx <= Kx; ++dx) {
                    const int xx = (cx + dx + 8 * D.nx) % D.nx;
                    const int yy = (cy + dy + 8 * D.ny) % D.ny;
                    const int zz = (cz + dz + 8 * D.nz) % D.nz;
                    const uint32_t c = D.cell0 + ((uint32_t)zz * D.ny + yy) * D.nx + xx;
                    const int b = (int)cell_start[c], e = (int)cell_start[c + 1];
                    for (int u = max(b, t + 1); u < e; ++u) {
                        const typename P::vec4 pj = pos[u];
                        double d[3];
                        if (P::kOffsets) {
                            d[0] = ((double)pi.x - (double)pj.x) + (double)(-dx) * D.h[0];
                            d[1] = ((double)pi.y - (double)pj.y) + (double)(-dy) * D.h[1];
                            d[2] = ((double)pi.z - (double)pj.z) + (double)(-dz) * D.h[2];
                        } else {
                            const double pa[3] = {(double)pi.x, (double)pi.y, (double)pi.z};
                            const double pb[3] = {(double)pj.x, (double)pj.y, (double)pj.z};
#pragma unroll
                            for (int q = 0; q < 3; ++q) {
                                const double dd = __dsub_rn(pa[q], pb[q]);
                                d[q] = __dsub_rn(dd, __dmul_rn(D.L[q], rint(__ddiv_rn(dd, D.L[q]))));
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

// --------------------------------------------------------------------------
// Re-packing after a system left: every surviving bead moves from its old
// slot (old bead0 of its system + its rank) to the new packed slot.
// --------------------------------------------------------------------------
template <class P>
struct RelayoutArgs {
    using vec4 = typename P::vec4;
    int n_new;
    const int *bsys_new;
    const SysDesc<P> *sys_new;
    const int *old_bead0;      // per system slot
    const vec4 *pos, *vel, *frc;
    const uint32_t *key;
    const int32_t *id;
    vec4 *pos_out, *vel_out, *frc_out;
    uint32_t *key_out;
    int32_t *id_out;
};

template <class P>
__global__ void __launch_bounds__(256) k_relayout(RelayoutArgs<P> a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_new) return;
    const int s = a.bsys_new[t];
    const int u = a.old_bead0[s] + (t - a.sys_new[s].bead0);
    a.pos_out[t] = a.pos[u];
    a.vel_out[t] = a.vel[u];
    a.frc_out[t] = a.frc[u];
    a.key_out[t] = a.key[u];
    a.id_out[t] = a.id[u];
}

}  // namespace dpd
