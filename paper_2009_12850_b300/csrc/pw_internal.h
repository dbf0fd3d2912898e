// pw_internal.h -- shared host/device definitions of the PW advection library.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pwadv.h"

// ---------------------------------------------------------------------------
// host-side objects
// ---------------------------------------------------------------------------
struct pw_mesh {
    int nx, ny, nz;
    int nzp;                 // padded column length (elements), multiple of 8
    int64_t sj, si, total;   // strides / total count in elements
    double dx, dy, tcx, tcy;
    pw_dtype dtype;
    pw_algo algo;
    int device;
    int num_sms;
    double *coef64;          // device, 12*nz: dz zf zn dzn rho_n rho_w tzc1 tzc2 tzd1 tzd2 Wuv Ww
    float *coef32;           // device, 4*nz: tzc1 tzc2 tzd1 tzd2
    float *coefsplit;        // device, 8*(nz+4)+4: float pairs of g, g', r, r' (levels -2..nz+1), tcx, tcy
    double *partials;        // device, residual scratch: PW_RED_SCRATCH doubles (zeroed at creation)
    double *host_sums;       // pinned host, PW_RED_STRIDE doubles: where the totals land
    int *status;             // device: [0] timeout status (0 or PW_ERR_TIMEOUT), [1] lid flag,
                             // [2] split-range flag, [3] unused
    int tile_j, tile_i;      // stencil tile: rows per CTA, columns marched per CTA
    int tile_i_auto;         // 1 while tile_i is the default (not set by the caller or the autotuner)
};

// words of the mesh status array
#define PW_STATUS_WORDS 4
#define PW_STATUS_RANGE_WORD 2  // set by the split kernels when a value was outside their range

// reduction geometry of pw_residuals (fixed so the order of sums is fixed):
// PW_RED_BLOCKS blocks each write PW_RED_STRIDE doubles (the 12 sums and a
// count of values outside the fast path's range), then PW_RED_STRIDE totals
// (written by the last block to finish), then one word counting the finished
// blocks (0 between calls)
#define PW_RED_BLOCKS 592
#define PW_RED_THREADS 256
#define PW_RED_FAST_THREADS 128
#define PW_RED_STRIDE 13
#define PW_RED_SCRATCH ((PW_RED_BLOCKS + 1) * PW_RED_STRIDE + 1)

// bounded waits: ~1 s at 2 GHz for a copy the kernel needs; ~50 ms when a
// kernel that already gave up drains copies still in flight.  On expiry the
// kernel records PW_ERR_TIMEOUT in the mesh status word, which is sticky: CTAs
// that start after it is set return at once, until the host clears it.
#define PW_WAIT_CYCLES (2000000000LL)
#define PW_DRAIN_CYCLES (100000000LL)

// error helpers (pw_mesh.cu)
pw_status pw_fail(pw_status st, const char *fmt, ...);
pw_status pw_cuda_fail(cudaError_t e, const char *what);
#define PW_CUDA(call)                                               \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return pw_cuda_fail(e_, #call);      \
    } while (0)

int pw_elem_in(pw_dtype d);    // bytes per field element
int pw_elem_out(pw_dtype d);   // bytes per source element
pw_status pw_check_ptr(const void *p, const char *name);

// TMA descriptor for one field of a mesh: box {kbox, rows, 1} over dims
// {kdim, ny+4, nx+4} with row stride nzp elements.  kdim is the number of
// levels the stencil may see: nz for u, v and their gradients, nz-1 for w and
// its gradient (the lid reads as 0); at least 1.
pw_status pw_make_field_map(CUtensorMap *map, const void *base, pw_dtype dtype, int nx, int ny,
                            int nzp, int kdim, int kbox, int rows);
static inline int pw_kdim(int nz, int field) { return field == 2 ? (nz > 1 ? nz - 1 : 1) : nz; }

// Columns marched per CTA for a launch whose other grid dimensions hold
// `ctas_per_column_tile` CTAs: the requested tile_i, halved (down to 4) while
// the grid would not fill one wave of the GPU (small domains would otherwise
// leave SMs idle and march long columns serially).
static inline int pw_fit_tile_i(const pw_mesh *m, int tile_i, long ctas_per_column_tile) {
    const long wave = 4L * m->num_sms;  // typical resident CTAs of the x-march kernels
    while (tile_i > 4 && ctas_per_column_tile * ((m->nx + tile_i - 1) / tile_i) < wave) tile_i = (tile_i + 1) / 2;
    return tile_i;
}

// Columns marched per CTA for an x-march launch of `tiles` CTAs per column
// range, `slots` of which fit on the GPU at once (resident CTAs per SM x SMs),
// each marching ti columns plus `prime` priming planes.  With the mesh's
// default tile the count in [4, 2 tile_i] that minimises the launch time when
// the CTAs run in waves: ceil(ctas / slots) waves, each as long as one CTA's
// march (the longer count wins ties: fewer priming planes in all), so a grid
// never ends in a nearly empty wave.  A tile set by the caller (or the
// autotuner) keeps pw_fit_tile_i's rule.
static inline int pw_pick_tile_i(const pw_mesh *m, int tile_i, long tiles, long slots, int prime) {
    if (!m->tile_i_auto || slots < 1 || tiles < 1) return pw_fit_tile_i(m, tile_i, tiles);
    const int hi = m->nx < 2 * tile_i ? m->nx : 2 * tile_i;
    int lo = hi < 4 ? hi : 4;
    while ((m->nx + lo - 1) / lo > 65535) lo++;  // grid dimension limit
    int best = hi > lo ? hi : lo;
    long long bestc = -1;
    for (int ti = best; ti >= lo; ti--) {
        const long long ctas = (long long)tiles * ((m->nx + ti - 1) / ti);
        const long long c = ((ctas + slots - 1) / slots) * (ti + prime);
        if (bestc < 0 || c < bestc) {
            bestc = c;
            best = ti;
        }
    }
    return best;
}

// resident CTAs of a kernel on the whole GPU (0 if the query fails)
template <typename K>
static inline long pw_slots(const pw_mesh *m, K kern, int threads, size_t smem) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (long)occ * m->num_sms;
}

// launchers (pw_advect.cu / pw_adjoint.cu)
pw_status pw_launch_advect(const pw_mesh *m, const void *u, const void *v, const void *w,
                           void *su, void *sv, void *sw, int beta, cudaStream_t st,
                           int tile_j, int tile_i);
pw_status pw_launch_step(const pw_mesh *m, const void *u, const void *v, const void *w, void *un, void *vn,
                         void *wn, double dt, cudaStream_t st, int tile_j, int tile_i);
pw_status pw_launch_advect_scalars(const pw_mesh *m, const void *u, const void *v, const void *w, int n,
                                   const void *const *phi, void *const *sphi, int beta, cudaStream_t st,
                                   int tile_j, int tile_i, int group);
pw_status pw_launch_halo(const pw_mesh *m, void *const *f, int nf, cudaStream_t st);
// ULTIMATE-QUICKEST for FP64 meshes in double-float arithmetic (pw_tvd_split.cu)
pw_status pw_launch_tvd_split(const pw_mesh *m, const void *u, const void *v, const void *w, int n,
                              const void *const *phi, void *const *sphi, double dt, int beta, cudaStream_t st);
// FP64 adjoint in double-float arithmetic (pw_adjoint_split.cu): in = u, v, w,
// gsu, gsv, gsw (halos of the gradients filled), out = gu, gv, gw.
pw_status pw_launch_adjoint_split(const pw_mesh *m, const void *const *in, void *const *out, double alpha,
                                  int beta, int add_y, cudaStream_t st);

// The conservation sums (pw_residuals.cu): the 12 sums into the HOST array
// out, computed on `st` with `scratch` (PW_RED_SCRATCH device doubles whose
// last word is 0) and the energy weights wuv, ww (device, nz each); the
// totals are copied through `staging` (PW_RED_STRIDE pinned host doubles, or
// NULL); synchronises `st`.
pw_status pw_residuals_run(int nx, int ny, int nz, int nzp, pw_dtype dtype, const double *wuv,
                           const double *ww, const void *u, const void *v, const void *w,
                           const void *su, const void *sv, const void *sw, double *scratch,
                           double *staging, double *out, cudaStream_t st);

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

__device__ __forceinline__ uint32_t pw_smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void pw_mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(pw_smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void pw_mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(pw_smem_u32(bar)) : "memory");
}

// order this thread's generic-proxy writes to shared memory before later
// asynchronous-proxy (TMA) writes to the same bytes
__device__ __forceinline__ void pw_fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void pw_fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void pw_mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(pw_smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// try_wait with a suspend-time hint: a waiting thread sleeps in hardware (up to
// ~0.1 ms per call) instead of spinning on the issue slots.
__device__ __forceinline__ bool pw_mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(pw_smem_u32(bar)), "r"(parity), "r"(100000u)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of an mbarrier with a cycle limit.  Returns false on
// expiry (the caller records PW_ERR_TIMEOUT and leaves).
__device__ __forceinline__ bool pw_mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                     long long limit = PW_WAIT_CYCLES) {
    if (pw_mbar_try_wait(bar, parity)) return true;
    long long t0 = clock64();
    while (!pw_mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

// true when an earlier CTA (or launch) on this status word has timed out
__device__ __forceinline__ bool pw_status_failed(const int *status) {
    return *reinterpret_cast<const volatile int *>(status) != 0;
}

// The same test taken once per CTA: thread 0 reads the word and shares the
// answer, so every thread takes the same branch (a CTA whose threads left at
// different points could no longer meet at a later barrier).  Contains CTA
// barriers: call it from every thread of the CTA.
__device__ __forceinline__ bool pw_cta_failed(const int *status) {
    __shared__ int flag;
    if (threadIdx.x == 0) flag = pw_status_failed(status);
    __syncthreads();
    const bool f = flag != 0;
    __syncthreads();  // the next call may overwrite the flag
    return f;
}

__device__ __forceinline__ void pw_tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1,
                                               int c2, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(pw_smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(pw_smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void pw_prefetch_map(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// scalar conversions of the storage types to the compute type
template <typename TC>
__device__ __forceinline__ TC pw_to(double x) { return (TC)x; }
template <typename TC>
__device__ __forceinline__ TC pw_to(float x) { return (TC)x; }
template <typename TC>
__device__ __forceinline__ TC pw_to(__nv_bfloat16 x) { return (TC)__bfloat162float(x); }

#endif  // __CUDACC__
