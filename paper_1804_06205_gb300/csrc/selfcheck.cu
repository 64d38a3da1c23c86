// Self-checks of the device code that tests call through the C ABI.
//
// dpd_wait_check: failure detection of the bounded device waits, exercised
// without a fault.  One block waits on an mbarrier with the same bounded poll
// loop as the pair kernel's staging wait.  With deliver = 1 a bulk copy brings
// the 16 bytes the barrier expects and the phase completes; with deliver = 0
// nothing is copied, the phase can never complete, the wait gives up after
// `tries` polls and the block records ST_TIMEOUT and returns.  No copy is ever
// left in flight, so the context stays usable.  The source and the status word
// are file-scope device variables: the call allocates nothing.
//
// dpd_grid_wait_check: the same for the grid-wide barrier of the persistent
// step kernel.  A small cooperative grid meets at one barrier that expects
// either exactly the grid (it completes) or one block more (nobody can
// complete it: every block gives up after its clock budget and records
// ST_TIMEOUT).  The barrier words and the status are file-scope device
// variables, cleared before the launch.
//
// dpd_bm_check: the FP64 Box-Muller logarithm and cosine (m2ln_u24 halved, cos_u24)
// against the library's log and cospi over all 2^23 uniforms n 2^-24; returns
// the largest absolute differences.
#include <cuda_runtime.h>

#include <cstring>

#include "dpd.h"
#include "kernels.cuh"
#include "persist.cuh"

namespace {

static __device__ __align__(16) unsigned char g_wc_src[16];
static __device__ int g_wc_status;
static __device__ dpd::GridBar g_gw_bar;
static __device__ int g_gw_status;

__global__ void k_wait_check(int deliver, int tries) {
    __shared__ __align__(16) unsigned char buf[16];
    __shared__ __align__(8) uint64_t mbar;
    if (threadIdx.x == 0) {
        dpd::mbar_init(&mbar, 1);
        dpd::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        dpd::mbar_expect_tx(&mbar, 16u);
        if (deliver) dpd::bulk_g2s(buf, g_wc_src, 16u, &mbar);
        dpd::mbar_arrive(&mbar);
    }
    const bool got = dpd::mbar_wait_bounded(&mbar, 0u, tries);
    if (__syncthreads_or(!got)) {
        if (threadIdx.x == 0) atomicOr(&g_wc_status, dpd::ST_TIMEOUT);
        return;
    }
    if (threadIdx.x == 0 && buf[0] != g_wc_src[0]) atomicOr(&g_wc_status, dpd::ST_BADINPUT);
}

// |-m2ln_u24(n) / 2 - log(n 2^-24)| and |cos_u24(n) - cospi(2 n 2^-24)| over every odd
// n < 2^24, their maxima kept as the bits of non-negative doubles (which order
// like the doubles)
__global__ void k_bm_check(const dpd::LnTab *t, unsigned long long *max_abs) {
    double ml = 0.0, mc = 0.0;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < (1u << 23);
         k += gridDim.x * blockDim.x) {
        const uint32_t n = 2u * k + 1u;
        const double u = (double)n * 0x1p-24;
        ml = fmax(ml, fabs(-0.5 * dpd::m2ln_u24(n, t) - log(u)));
        mc = fmax(mc, fabs(dpd::cos_u24(n) - cospi(2.0 * u)));
    }
    atomicMax(max_abs, (unsigned long long)__double_as_longlong(ml));
    atomicMax(max_abs + 1, (unsigned long long)__double_as_longlong(mc));
}

}  // namespace

extern "C" int dpd_bm_check(double *ln_err, double *cos_err) {
    if (!ln_err || !cos_err) return DPD_EINVAL;
    dpd::LnTab *t = nullptr;
    unsigned long long *m = nullptr, mh[2] = {0, 0};
    int rc = DPD_OK;
    if (cudaMalloc(&t, sizeof(dpd::LnTab)) != cudaSuccess ||
        cudaMalloc(&m, 2 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(m, 0, 2 * sizeof(unsigned long long)) != cudaSuccess) {
        rc = DPD_ECUDA;
    } else {
        dpd::k_ln_tab<<<1, 128>>>(t);
        k_bm_check<<<1024, 256>>>(t, m);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(mh, m, sizeof(mh), cudaMemcpyDeviceToHost) != cudaSuccess) {
            rc = DPD_ECUDA;
        } else {
            std::memcpy(ln_err, &mh[0], sizeof(double));
            std::memcpy(cos_err, &mh[1], sizeof(double));
        }
    }
    if (t) cudaFree(t);
    if (m) cudaFree(m);
    return rc;
}

extern "C" int dpd_wait_check(int32_t deliver, int32_t tries, void *cuda_stream) {
    if (tries <= 0 || tries > DPD_WAIT_CHECK_MAX_TRIES) return DPD_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int zero = 0;
    if (cudaMemcpyToSymbolAsync(g_wc_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return DPD_ECUDA;
    k_wait_check<<<1, 32, 0, st>>>(deliver ? 1 : 0, tries);
    if (cudaGetLastError() != cudaSuccess) return DPD_ECUDA;
    int status = 0;
    if (cudaMemcpyFromSymbolAsync(&status, g_wc_status, sizeof(int), 0, cudaMemcpyDeviceToHost,
                                  st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return DPD_ECUDA;
    if (status & dpd::ST_TIMEOUT) return DPD_ETIMEOUT;
    return status ? DPD_ECUDA : DPD_OK;
}

extern "C" int dpd_grid_wait_check(int32_t complete, int64_t budget_cycles, void *cuda_stream) {
    if (budget_cycles <= 0 || budget_cycles > DPD_GRID_WAIT_CHECK_MAX_CYCLES) return DPD_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const dpd::GridBar zb = {0u, 0u};
    const int zero = 0;
    if (cudaMemcpyToSymbolAsync(g_gw_bar, &zb, sizeof(zb), 0, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyToSymbolAsync(g_gw_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
        return DPD_ECUDA;
    dpd::GridBar *bar = nullptr;
    int *status = nullptr;
    if (cudaGetSymbolAddress((void **)&bar, g_gw_bar) != cudaSuccess ||
        cudaGetSymbolAddress((void **)&status, g_gw_status) != cudaSuccess)
        return DPD_ECUDA;
    constexpr unsigned int kGrid = 4;   // co-resident on any GPU
    const unsigned int expect = complete ? kGrid : kGrid + 1;
    const long long budget = (long long)budget_cycles;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kGrid);
    cfg.blockDim = dim3(64);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, dpd::k_grid_wait_check, bar, expect, budget, status) != cudaSuccess)
        return DPD_ECUDA;
    int out = 0;
    if (cudaMemcpyFromSymbolAsync(&out, g_gw_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return DPD_ECUDA;
    if (out & dpd::ST_TIMEOUT) return DPD_ETIMEOUT;
    return out ? DPD_ECUDA : DPD_OK;
}
