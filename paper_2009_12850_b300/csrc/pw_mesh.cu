// pw_mesh.cu -- mesh set-up, coefficients (FP64 on the GPU), periodic halo
// fill, forward-Euler update with halo refresh, conservation reductions and
// the error plumbing of the C-ABI.
#include <math.h>

#include <algorithm>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "pw_internal.h"

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local char g_last_error[512] = "";

pw_status pw_fail(pw_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return st;
}

pw_status pw_cuda_fail(cudaError_t e, const char *what) {
    return pw_fail(PW_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

extern "C" const char *pw_last_error(void) { return g_last_error; }

extern "C" const char *pw_status_string(pw_status s) {
    switch (s) {
        case PW_OK: return "ok";
        case PW_ERR_ARG: return "invalid argument";
        case PW_ERR_SHAPE: return "shape mismatch or out of range";
        case PW_ERR_ALIGN: return "buffer not 16-byte aligned";
        case PW_ERR_DTYPE: return "operation not available for this dtype";
        case PW_ERR_LID: return "non-zero lid value";
        case PW_ERR_CUDA: return "CUDA error";
        case PW_ERR_TIMEOUT: return "device wait timed out";
        case PW_ERR_NOMEM: return "out of memory";
        case PW_ERR_IO: return "autotune cache i/o error";
        case PW_ERR_RANGE: return "value outside the range of the split FP64 arithmetic";
    }
    return "unknown status";
}

extern "C" int pw_version(void) { return PWADV_VERSION; }

int pw_elem_in(pw_dtype d) { return d == PW_F64 ? 8 : d == PW_F32 ? 4 : 2; }
int pw_elem_out(pw_dtype d) { return d == PW_F64 ? 8 : d == PW_BF16_OUT ? 2 : 4; }

pw_status pw_check_ptr(const void *p, const char *name) {
    if (!p) return pw_fail(PW_ERR_ARG, "%s is NULL", name);
    if (((uintptr_t)p) & 15u) return pw_fail(PW_ERR_ALIGN, "%s is not 16-byte aligned", name);
    return PW_OK;
}

// ---------------------------------------------------------------------------
// TMA descriptors
// ---------------------------------------------------------------------------
typedef CUresult (*pw_encode_tiled_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                       const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                       const cuuint32_t *, CUtensorMapInterleave,
                                       CUtensorMapSwizzle, CUtensorMapL2promotion,
                                       CUtensorMapFloatOOBfill);

static pw_encode_tiled_fn pw_encoder() {
    static pw_encode_tiled_fn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (pw_encode_tiled_fn)p;
    }
    return fn;
}

pw_status pw_make_field_map(CUtensorMap *map, const void *base, pw_dtype dtype, int nx, int ny,
                            int nzp, int kdim, int kbox, int rows) {
    pw_encode_tiled_fn enc = pw_encoder();
    if (!enc) return pw_fail(PW_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    int es = pw_elem_in(dtype);
    CUtensorMapDataType dt = dtype == PW_F64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                             : dtype == PW_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                               : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    // the k extent is the logical one (nz, or nz-1 for w) while the row stride
    // stays nzp: TMA fills levels beyond it with 0, which is how the padding and
    // the lid face of w reach the stencil as zeros
    cuuint64_t dims[3] = {(cuuint64_t)kdim, (cuuint64_t)(ny + 4), (cuuint64_t)(nx + 4)};
    cuuint64_t strides[2] = {(cuuint64_t)nzp * es, (cuuint64_t)nzp * es * (ny + 4)};
    cuuint32_t box[3] = {(cuuint32_t)kbox, (cuuint32_t)rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, dt, 3, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return pw_fail(PW_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d): box %u x %u, nzp %d",
                       (int)r, box[0], box[1], nzp);
    return PW_OK;
}

// ---------------------------------------------------------------------------
// A1: vertical grid and coefficients in FP64, one CTA, levels in parallel.
// zf(k) is summed by thread k over dz(0..k) in increasing order, so every
// prefix is rounded exactly as a sequential running sum would round it.
// ---------------------------------------------------------------------------
__global__ void pw_coeffs_kernel(int nz, const double *dz_in, const double *rn_in,
                                 const double *rw_in, int have_dz, int have_rn, int have_rw,
                                 double rho0, double H, double *c64, float *c32) {
    if (blockIdx.x != 0) return;
    double *dz = c64, *zf = c64 + nz, *zn = c64 + 2 * nz, *dzn = c64 + 3 * nz;
    double *rn = c64 + 4 * nz, *rw = c64 + 5 * nz;
    double *t1 = c64 + 6 * nz, *t2 = c64 + 7 * nz, *d1 = c64 + 8 * nz, *d2 = c64 + 9 * nz;
    double *wuv = c64 + 10 * nz, *ww = c64 + 11 * nz;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        if (have_dz) dz[k] = dz_in[k];
        else if (nz == 1) dz[k] = 10.0;
        else dz[k] = 10.0 * pow(4.0, (double)k / (double)(nz - 1));
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        double z = 0.0;
        for (int q = 0; q <= k; q++) z += dz[q];
        zf[k] = z;
        zn[k] = z - 0.5 * dz[k];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        dzn[k] = (k < nz - 1) ? zn[k + 1] - zn[k] : 0.0;
        rn[k] = have_rn ? rn_in[k] : rho0 * exp(-zn[k] / H);
        rw[k] = have_rw ? rw_in[k] : rho0 * exp(-zf[k] / H);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        double below = (k == 0) ? rho0 : rw[k - 1];
        t1[k] = 0.25 * below / (rn[k] * dz[k]);
        t2[k] = 0.25 * rw[k] / (rn[k] * dz[k]);
        if (k < nz - 1) {
            d1[k] = 0.25 * rn[k] / (rw[k] * dzn[k]);
            d2[k] = 0.25 * rn[k + 1] / (rw[k] * dzn[k]);
        } else {
            d1[k] = 0.0;
            d2[k] = 0.0;
        }
        wuv[k] = rn[k] * dz[k];
        ww[k] = (k < nz - 1) ? rw[k] * dzn[k] : 0.0;
        c32[k] = (float)t1[k];
        c32[nz + k] = (float)t2[k];
        c32[2 * nz + k] = (float)d1[k];
        c32[3 * nz + k] = (float)d2[k];
    }
}

// Float-pair table for the FP64 split kernel: the vertical coefficients are
// regrouped as tzc1(k) = g(k-1) r(k), tzc2(k) = g(k) r(k), tzd1(k) = g'(k) r'(k),
// tzd2(k) = g'(k+1) r'(k) with g = 0.25 rho_w, g' = 0.25 rho_n, r = 1/(rho_n dz),
// r' = 1/(rho_w dzn) (0 on the lid face), each stored as hi + lo floats for
// levels -2 .. nz+1 (0 outside 0..nz-1), followed by tcx and tcy.
__global__ void pw_coeffs_split_kernel(int nz, const double *c64, double tcx, double tcy, float *cs) {
    if (blockIdx.x != 0) return;
    const double *dz = c64, *dzn = c64 + 3 * nz, *rn = c64 + 4 * nz, *rw = c64 + 5 * nz;
    const int n = nz + 4;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int k = q - 2;
        const bool in = k >= 0 && k < nz;
        double v[4];
        v[0] = in ? 0.25 * rw[k] : 0.0;
        v[1] = in ? 0.25 * rn[k] : 0.0;
        v[2] = in ? 1.0 / (rn[k] * dz[k]) : 0.0;
        v[3] = (in && k < nz - 1) ? 1.0 / (rw[k] * dzn[k]) : 0.0;
        for (int a = 0; a < 4; a++) {
            const float h = (float)v[a];
            cs[(2 * a) * n + q] = h;
            cs[(2 * a + 1) * n + q] = (float)(v[a] - (double)h);
        }
    }
    if (threadIdx.x != 0) return;
    const double t[2] = {tcx, tcy};
    for (int a = 0; a < 2; a++) {
        const float h = (float)t[a];
        cs[8 * n + 2 * a] = h;
        cs[8 * n + 2 * a + 1] = (float)(t[a] - (double)h);
    }
}

static void pw_mesh_free(pw_mesh *m) {
    if (!m) return;
    cudaFree(m->coef64);
    cudaFree(m->coef32);
    cudaFree(m->coefsplit);
    cudaFree(m->partials);
    cudaFreeHost(m->host_sums);
    cudaFree(m->status);
    free(m);
}

extern "C" pw_status pw_mesh_create(const pw_mesh_desc *d, void *stream, pw_mesh **out) {
    if (!d || !out) return pw_fail(PW_ERR_ARG, "desc and out must not be NULL");
    *out = nullptr;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || d->nz > PW_MAX_NZ)
        return pw_fail(PW_ERR_SHAPE, "bad sizes nx=%d ny=%d nz=%d (need >= 1, nz <= %d)", d->nx,
                       d->ny, d->nz, PW_MAX_NZ);
    if ((int64_t)(d->nx + 4) * (d->ny + 4) > (int64_t)1 << 31 || d->nx > 1 << 20 || d->ny > 1 << 20)
        return pw_fail(PW_ERR_SHAPE, "horizontal size too large");
    if (!(d->dx > 0) || !(d->dy > 0)) return pw_fail(PW_ERR_ARG, "dx and dy must be > 0");
    if (d->dtype != PW_F64 && d->dtype != PW_F32 && d->dtype != PW_BF16 && d->dtype != PW_BF16_OUT)
        return pw_fail(PW_ERR_DTYPE, "unknown dtype %d", (int)d->dtype);
    if (d->algo < PW_ALGO_AUTO || d->algo > PW_ALGO_F64_SPLIT)
        return pw_fail(PW_ERR_ARG, "unknown algo %d", (int)d->algo);
    double rho0 = d->rho0, H = d->H_rho;
    if (rho0 == 0.0 && H == 0.0) {
        rho0 = 1.2;
        H = 8000.0;
    }
    if (!(rho0 > 0) || H == 0.0) return pw_fail(PW_ERR_ARG, "rho0 must be > 0 and H_rho != 0");
    int nz = d->nz;
    for (int k = 0; d->dz && k < nz; k++)
        if (!(d->dz[k] > 0)) return pw_fail(PW_ERR_ARG, "dz[%d] must be > 0", k);
    for (int k = 0; d->rho_n && k < nz; k++)
        if (!(d->rho_n[k] > 0)) return pw_fail(PW_ERR_ARG, "rho_n[%d] must be > 0", k);
    for (int k = 0; d->rho_w && k < nz; k++)
        if (!(d->rho_w[k] > 0)) return pw_fail(PW_ERR_ARG, "rho_w[%d] must be > 0", k);

    pw_mesh *m = (pw_mesh *)calloc(1, sizeof(pw_mesh));
    if (!m) return pw_fail(PW_ERR_NOMEM, "host allocation");
    m->nx = d->nx;
    m->ny = d->ny;
    m->nz = nz;
    m->nzp = (nz + 7) / 8 * 8;
    m->sj = m->nzp;
    m->si = (int64_t)(d->ny + 4) * m->nzp;
    m->total = (int64_t)(d->nx + 4) * m->si;
    m->dx = d->dx;
    m->dy = d->dy;
    m->tcx = 0.25 / d->dx;
    m->tcy = 0.25 / d->dy;
    m->dtype = d->dtype;
    m->algo = d->algo == PW_ALGO_AUTO ? PW_ALGO_F64_SPLIT : d->algo;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&m->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device);
    if (e != cudaSuccess) {
        pw_mesh_free(m);
        return pw_cuda_fail(e, "device query");
    }
    // defaults from timing on B300 at 1024 x 1024 x 128 (pw_autotune refines
    // them): the double-float kernels run 8 rows x 32-level chunks per CTA
    m->tile_j = (m->dtype == PW_F64 && m->algo == PW_ALGO_F64_SPLIT) ? 8 : 4;
    m->tile_i = 64;
    m->tile_i_auto = 1;
    double *tmp = nullptr;
    if ((e = cudaMalloc(&m->coef64, 12 * (size_t)nz * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&m->coef32, 4 * (size_t)nz * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&m->coefsplit, (8 * ((size_t)nz + 4) + 4) * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&m->partials, PW_RED_SCRATCH * sizeof(double))) != cudaSuccess ||
        (e = cudaMemset(m->partials, 0, PW_RED_SCRATCH * sizeof(double))) != cudaSuccess ||
        (e = cudaHostAlloc(&m->host_sums, PW_RED_STRIDE * sizeof(double), cudaHostAllocDefault)) != cudaSuccess ||
        (e = cudaMalloc(&m->status, PW_STATUS_WORDS * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&tmp, 3 * (size_t)nz * sizeof(double))) != cudaSuccess) {
        pw_mesh_free(m);
        cudaFree(tmp);
        return pw_cuda_fail(e, "cudaMalloc (mesh)");
    }
    pw_status rs = PW_OK;
    do {
        if (d->dz && (e = cudaMemcpyAsync(tmp, d->dz, nz * sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
        if (d->rho_n && (e = cudaMemcpyAsync(tmp + nz, d->rho_n, nz * sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
        if (d->rho_w && (e = cudaMemcpyAsync(tmp + 2 * nz, d->rho_w, nz * sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(m->status, 0, PW_STATUS_WORDS * sizeof(int), st)) != cudaSuccess) break;
        pw_coeffs_kernel<<<1, 256, 0, st>>>(nz, tmp, tmp + nz, tmp + 2 * nz, d->dz != nullptr,
                                           d->rho_n != nullptr, d->rho_w != nullptr, rho0, H,
                                           m->coef64, m->coef32);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        pw_coeffs_split_kernel<<<1, 256, 0, st>>>(nz, m->coef64, m->tcx, m->tcy, m->coefsplit);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        e = cudaStreamSynchronize(st);
    } while (0);
    cudaFree(tmp);
    if (e != cudaSuccess) {
        pw_mesh_free(m);
        return pw_cuda_fail(e, "mesh coefficient set-up");
    }
    // sanity: the coefficients must be finite
    double *h = (double *)malloc(12 * (size_t)nz * sizeof(double));
    if (!h) {
        pw_mesh_free(m);
        return pw_fail(PW_ERR_NOMEM, "host allocation");
    }
    e = cudaMemcpy(h, m->coef64, 12 * (size_t)nz * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rs = pw_cuda_fail(e, "coefficient read-back");
    for (int q = 0; rs == PW_OK && q < 12 * nz; q++)
        if (!isfinite(h[q])) rs = pw_fail(PW_ERR_ARG, "non-finite vertical coefficient (check dz/rho)");
    // the split arithmetic needs tcx, tcy and the vertical coefficients in
    // [2^-16, 2^8] and the density factors 0.25 rho in [2^-36, 2^24] (its
    // intermediate products then stay inside the FP32 range); PW_ALGO_AUTO falls
    // back to native FP64 outside that range, PW_ALGO_F64_SPLIT is refused
    if (rs == PW_OK && m->dtype == PW_F64 && m->algo == PW_ALGO_F64_SPLIT) {
        const double *rn = h + 4 * nz, *rw = h + 5 * nz, *tz = h + 6 * nz;
        auto out_of = [](double x, int lo, int hi) { return !(x >= ldexp(1.0, lo) && x <= ldexp(1.0, hi)); };
        bool bad = out_of(m->tcx, -16, 8) || out_of(m->tcy, -16, 8);
        for (int k = 0; k < nz && !bad; k++) {
            bad = out_of(0.25 * rw[k], -36, 24) || out_of(0.25 * rn[k], -36, 24);
            // tzc1 tzc2 tzd1 tzd2 (tzd 0 on the lid face; tzc1 at k = 0 multiplies
            // the ground face, w = 0, and is not used)
            for (int a = (k == 0 ? 1 : 0); a < 4 && !bad; a++)
                bad = tz[a * nz + k] != 0.0 && out_of(tz[a * nz + k], -16, 8);
        }
        if (bad && d->algo == PW_ALGO_F64_SPLIT)
            rs = pw_fail(PW_ERR_RANGE, "mesh coefficients outside the split range (tcx, tcy, tzc, tzd in "
                                       "[2^-16, 2^8], 0.25 rho in [2^-36, 2^24]): use PW_ALGO_F64_NATIVE");
        else if (bad) {
            m->algo = PW_ALGO_F64_NATIVE;
            m->tile_j = 4;
        }
    }
    free(h);
    if (rs != PW_OK) {
        pw_mesh_free(m);
        return rs;
    }
    *out = m;
    return PW_OK;
}

extern "C" void pw_mesh_destroy(pw_mesh *m) { pw_mesh_free(m); }

extern "C" pw_status pw_mesh_layout(const pw_mesh *m, int64_t *nzp, int64_t *sj, int64_t *si,
                                    int64_t *total) {
    if (!m) return pw_fail(PW_ERR_ARG, "mesh is NULL");
    if (nzp) *nzp = m->nzp;
    if (sj) *sj = m->sj;
    if (si) *si = m->si;
    if (total) *total = m->total;
    return PW_OK;
}

extern "C" pw_status pw_mesh_algo(const pw_mesh *m, pw_algo *out) {
    if (!m || !out) return pw_fail(PW_ERR_ARG, "mesh and out must not be NULL");
    *out = m->dtype == PW_F64 ? m->algo : PW_ALGO_AUTO;
    return PW_OK;
}

extern "C" pw_status pw_mesh_coefficients(const pw_mesh *m, double *out, double *out_h) {
    if (!m || !out) return pw_fail(PW_ERR_ARG, "mesh and out must not be NULL");
    PW_CUDA(cudaMemcpy(out, m->coef64, 12 * (size_t)m->nz * sizeof(double), cudaMemcpyDeviceToHost));
    if (out_h) {
        out_h[0] = m->tcx;
        out_h[1] = m->tcy;
    }
    return PW_OK;
}

extern "C" pw_status pw_mesh_device_status(const pw_mesh *m, int clear, void *stream, int *status) {
    if (!m || !status) return pw_fail(PW_ERR_ARG, "mesh and status must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int h[PW_STATUS_WORDS] = {0};
    PW_CUDA(cudaMemcpyAsync(h, m->status, sizeof(h), cudaMemcpyDeviceToHost, st));
    if (clear) {
        PW_CUDA(cudaMemsetAsync(m->status, 0, sizeof(int), st));
        PW_CUDA(cudaMemsetAsync(m->status + PW_STATUS_RANGE_WORD, 0, sizeof(int), st));
    }
    PW_CUDA(cudaStreamSynchronize(st));
    *status = h[0] != 0 ? h[0] : h[PW_STATUS_RANGE_WORD] != 0 ? (int)PW_ERR_RANGE : 0;
    return PW_OK;
}

extern "C" pw_status pw_mesh_set_tile(pw_mesh *m, int tile_j, int tile_i) {
    if (!m) return pw_fail(PW_ERR_ARG, "mesh is NULL");
    if (tile_j < 1 || tile_j > 32 || tile_i < 1 || tile_i > 1 << 20)
        return pw_fail(PW_ERR_ARG, "tile_j must be in 1..32 and tile_i >= 1");
    m->tile_j = tile_j;
    m->tile_i = tile_i;
    m->tile_i_auto = 0;
    return PW_OK;
}

extern "C" pw_status pw_mesh_get_tile(const pw_mesh *m, int *tile_j, int *tile_i) {
    if (!m) return pw_fail(PW_ERR_ARG, "mesh is NULL");
    if (tile_j) *tile_j = m->tile_j;
    if (tile_i) *tile_i = m->tile_i;
    return PW_OK;
}

// ---------------------------------------------------------------------------
// A2: periodic halo fill.  One warp per halo column; each lane copies 16-byte
// chunks of the column from its periodic image in the interior.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pw_wrap(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

__global__ void pw_halo_kernel(char *f0, char *f1, char *f2, int nx, int ny, int64_t col_bytes,
                               int64_t col_stride, int nchunk) {
    char *f = blockIdx.y == 0 ? f0 : blockIdx.y == 1 ? f1 : f2;
    int warps = blockDim.x >> 5;
    int64_t c = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    int64_t rows = 4LL * (ny + 4);      // full halo rows ih in {0,1,nx+2,nx+3}
    int64_t total = rows + 4LL * nx;    // plus side halos jh in {0,1,ny+2,ny+3}
    if (c >= total) return;
    int ih, jh;
    if (c < rows) {
        int r = (int)(c / (ny + 4));
        ih = r < 2 ? r : nx + r;
        jh = (int)(c % (ny + 4));
    } else {
        int64_t q = c - rows;
        ih = 2 + (int)(q / 4);
        int s = (int)(q % 4);
        jh = s < 2 ? s : ny + s;
    }
    int is = pw_wrap(ih - 2, nx) + 2, js = pw_wrap(jh - 2, ny) + 2;
    const int4 *src = reinterpret_cast<const int4 *>(f + ((int64_t)is * (ny + 4) + js) * col_stride);
    int4 *dst = reinterpret_cast<int4 *>(f + ((int64_t)ih * (ny + 4) + jh) * col_stride);
    for (int q = lane; q < nchunk; q += 32) dst[q] = src[q];
    (void)col_bytes;
}

pw_status pw_launch_halo(const pw_mesh *m, void *const *f, int nf, cudaStream_t st) {
    int es = pw_elem_in(m->dtype);
    int64_t col_stride = (int64_t)m->nzp * es;
    int64_t used = (int64_t)m->nz * es;
    int nchunk = (int)((used + 15) / 16);
    int64_t total = 4LL * (m->ny + 4) + 4LL * m->nx;
    int warps = 8;
    dim3 grid((unsigned)((total + warps - 1) / warps), (unsigned)nf);
    char *p0 = (char *)f[0];
    char *p1 = nf > 1 ? (char *)f[1] : p0;
    char *p2 = nf > 2 ? (char *)f[2] : p0;
    pw_halo_kernel<<<grid, warps * 32, 0, st>>>(p0, p1, p2, m->nx, m->ny, used, col_stride, nchunk);
    PW_CUDA(cudaGetLastError());
    return PW_OK;
}

extern "C" pw_status pw_halo_periodic(const pw_mesh *m, void *f1, void *f2, void *f3, void *stream) {
    if (!m) return pw_fail(PW_ERR_ARG, "mesh is NULL");
    pw_status s;
    if ((s = pw_check_ptr(f1, "f1")) != PW_OK) return s;
    void *f[3];
    int n = 0;
    f[n++] = f1;
    if (f2) {
        if ((s = pw_check_ptr(f2, "f2")) != PW_OK) return s;
        f[n++] = f2;
    }
    if (f3) {
        if ((s = pw_check_ptr(f3, "f3")) != PW_OK) return s;
        f[n++] = f3;
    }
    return pw_launch_halo(m, f, n, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// Adjoint of the periodic halo fill: every halo value is added onto the
// interior value it copies and the halo is zeroed.  Only interior columns
// within two of an x or y edge have halo images; one thread per element of
// those columns gathers from all its images, so there are no races.  The
// edge columns are enumerated directly: the nr edge rows (i < 2 or
// i >= nx - 2; all rows when nx <= 4) with every j, then the other rows with
// their nc edge columns (j < 2 or j >= ny - 2; all when ny <= 4).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pw_edge_index(int q, int n) {  // q-th of the indices < 2 or >= n - 2
    return n <= 4 ? q : (q < 2 ? q : n - 4 + q);
}

template <typename T>
__global__ void pw_halo_fold_kernel(T *f0, T *f1, T *f2, int nx, int ny, int nz, int nzp) {
    T *f = blockIdx.y == 0 ? f0 : blockIdx.y == 1 ? f1 : f2;
    const int nr = nx < 4 ? nx : 4, nc = ny < 4 ? ny : 4;
    const int64_t first = (int64_t)nr * ny;                 // columns of the edge rows
    const int64_t ncols = first + (int64_t)(nx - nr) * nc;  // plus the edge columns of the others
    const int64_t n = ncols * nz;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const int k = (int)(e % nz);
        const int64_t q = e / nz;
        int i, j;
        if (q < first) {
            i = pw_edge_index((int)(q / ny), nx);
            j = (int)(q % ny);
        } else {
            const int64_t r = q - first;
            i = 2 + (int)(r / nc);  // rows 2 .. nx-3 (nx > 4 here)
            j = pw_edge_index((int)(r % nc), ny);
        }
        T acc = T(0);
        for (int ih = i + 2 - ((i + 2) / nx) * nx; ih < nx + 4; ih += nx)
            for (int jh = j + 2 - ((j + 2) / ny) * ny; jh < ny + 4; jh += ny) {
                if (ih >= 2 && ih < nx + 2 && jh >= 2 && jh < ny + 2) continue;
                T *h = f + ((int64_t)ih * (ny + 4) + jh) * nzp + k;
                acc += *h;
                *h = T(0);
            }
        f[((int64_t)(i + 2) * (ny + 4) + (j + 2)) * nzp + k] += acc;
    }
}

extern "C" pw_status pw_halo_fold(const pw_mesh *m, void *f1, void *f2, void *f3, void *stream) {
    if (!m) return pw_fail(PW_ERR_ARG, "mesh is NULL");
    pw_status s;
    void *f[3] = {f1, f2, f3};
    const char *nm[3] = {"f1", "f2", "f3"};
    int n = 0;
    for (int q = 0; q < 3; q++) {
        if (q > 0 && !f[q]) continue;
        if ((s = pw_check_ptr(f[q], nm[q])) != PW_OK) return s;
        f[n++] = f[q];
    }
    if (m->dtype != PW_F64 && m->dtype != PW_F32)
        return pw_fail(PW_ERR_DTYPE, "pw_halo_fold supports PW_F64 and PW_F32 meshes");
    const long long nr = m->nx < 4 ? m->nx : 4, nc = m->ny < 4 ? m->ny : 4;
    const long long elems = (nr * m->ny + (long long)(m->nx - nr) * nc) * m->nz;
    const long long blocks = std::min<long long>((elems + 255) / 256, (long long)m->num_sms * 4);
    dim3 grid((unsigned)std::max<long long>(blocks, 1), (unsigned)n);
    cudaStream_t st = (cudaStream_t)stream;
    void *a = f[0], *b = n > 1 ? f[1] : f[0], *c = n > 2 ? f[2] : f[0];
    if (m->dtype == PW_F64)
        pw_halo_fold_kernel<double><<<grid, 256, 0, st>>>((double *)a, (double *)b, (double *)c, m->nx, m->ny, m->nz, m->nzp);
    else
        pw_halo_fold_kernel<float><<<grid, 256, 0, st>>>((float *)a, (float *)b, (float *)c, m->nx, m->ny, m->nz, m->nzp);
    PW_CUDA(cudaGetLastError());
    return PW_OK;
}

// ---------------------------------------------------------------------------
// forward Euler with halo refresh: each interior element is updated once and
// written to every halo column that is a periodic image of it.
// ---------------------------------------------------------------------------
template <typename T, typename TS>
__global__ void pw_euler_kernel(T *u, T *v, T *w, const TS *su, const TS *sv, const TS *sw,
                                int nx, int ny, int nz, int nzp, double dt) {
    T *x = blockIdx.y == 0 ? u : blockIdx.y == 1 ? v : w;
    const TS *s = blockIdx.y == 0 ? su : blockIdx.y == 1 ? sv : sw;
    int64_t n = (int64_t)nx * ny * nz;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        int k = (int)(e % nz);
        int64_t col = e / nz;
        int j = (int)(col % ny), i = (int)(col / ny);
        int64_t off = ((int64_t)(i + 2) * (ny + 4) + (j + 2)) * nzp + k;
        T val = (T)((double)x[off] + dt * (double)s[off]);
        x[off] = val;
        bool ei = (i < 2) || (i >= nx - 2), ej = (j < 2) || (j >= ny - 2);
        if (!ei && !ej) continue;
        // every halo column (ih, jh) whose periodic image is (i, j)
        for (int ih = i + 2 - ((i + 2) / nx) * nx; ih < nx + 4; ih += nx) {
            if (ih < 0) continue;
            for (int jh = j + 2 - ((j + 2) / ny) * ny; jh < ny + 4; jh += ny) {
                if (jh < 0) continue;
                if (ih >= 2 && ih < nx + 2 && jh >= 2 && jh < ny + 2) continue;  // interior
                x[((int64_t)ih * (ny + 4) + jh) * nzp + k] = val;
            }
        }
    }
}

// float path: update in FP32 (no double arithmetic)
template <>
__global__ void pw_euler_kernel<float, float>(float *u, float *v, float *w, const float *su,
                                              const float *sv, const float *sw, int nx, int ny,
                                              int nz, int nzp, double dtd) {
    float *x = blockIdx.y == 0 ? u : blockIdx.y == 1 ? v : w;
    const float *s = blockIdx.y == 0 ? su : blockIdx.y == 1 ? sv : sw;
    float dt = (float)dtd;
    int64_t n = (int64_t)nx * ny * nz;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        int k = (int)(e % nz);
        int64_t col = e / nz;
        int j = (int)(col % ny), i = (int)(col / ny);
        int64_t off = ((int64_t)(i + 2) * (ny + 4) + (j + 2)) * nzp + k;
        float val = fmaf(dt, s[off], x[off]);
        x[off] = val;
        bool ei = (i < 2) || (i >= nx - 2), ej = (j < 2) || (j >= ny - 2);
        if (!ei && !ej) continue;
        for (int ih = i + 2 - ((i + 2) / nx) * nx; ih < nx + 4; ih += nx) {
            if (ih < 0) continue;
            for (int jh = j + 2 - ((j + 2) / ny) * ny; jh < ny + 4; jh += ny) {
                if (jh < 0) continue;
                if (ih >= 2 && ih < nx + 2 && jh >= 2 && jh < ny + 2) continue;
                x[((int64_t)ih * (ny + 4) + jh) * nzp + k] = val;
            }
        }
    }
}

extern "C" pw_status pw_euler(const pw_mesh *m, void *u, void *v, void *w, const void *su,
                              const void *sv, const void *sw, double dt, void *stream) {
    if (!m) return pw_fail(PW_ERR_ARG, "mesh is NULL");
    pw_status s;
    const void *ps[6] = {u, v, w, su, sv, sw};
    const char *nm[6] = {"u", "v", "w", "su", "sv", "sw"};
    for (int q = 0; q < 6; q++)
        if ((s = pw_check_ptr(ps[q], nm[q])) != PW_OK) return s;
    if (!isfinite(dt)) return pw_fail(PW_ERR_ARG, "dt must be finite");
    cudaStream_t st = (cudaStream_t)stream;
    dim3 grid((unsigned)(m->num_sms * 4), 3);
    if (m->dtype == PW_F64)
        pw_euler_kernel<double, double><<<grid, 256, 0, st>>>(
            (double *)u, (double *)v, (double *)w, (const double *)su, (const double *)sv,
            (const double *)sw, m->nx, m->ny, m->nz, m->nzp, dt);
    else if (m->dtype == PW_F32)
        pw_euler_kernel<float, float><<<grid, 256, 0, st>>>(
            (float *)u, (float *)v, (float *)w, (const float *)su, (const float *)sv,
            (const float *)sw, m->nx, m->ny, m->nz, m->nzp, dt);
    else
        return pw_fail(PW_ERR_DTYPE, "pw_euler supports PW_F64 and PW_F32 meshes");
    PW_CUDA(cudaGetLastError());
    return PW_OK;
}

// ---------------------------------------------------------------------------
// failure-path self-test: a bounded wait on an mbarrier that nothing completes
// ---------------------------------------------------------------------------
__global__ void pw_selftest_timeout_kernel(int *status, long long cycles) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        pw_mbar_init(&bar, 1);
        pw_fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !pw_mbar_wait_bounded(&bar, 0, cycles)) atomicExch(status, (int)PW_ERR_TIMEOUT);
    __syncthreads();
    if (threadIdx.x == 0) pw_mbar_inval(&bar);
}

extern "C" pw_status pw_selftest_timeout(const pw_mesh *m, long long cycles, void *stream) {
    if (!m) return pw_fail(PW_ERR_ARG, "mesh is NULL");
    if (cycles < 1 || cycles > PW_WAIT_CYCLES) return pw_fail(PW_ERR_ARG, "cycles must be in 1..%lld", PW_WAIT_CYCLES);
    pw_selftest_timeout_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(m->status, cycles);
    PW_CUDA(cudaGetLastError());
    return PW_OK;
}

// ---------------------------------------------------------------------------
// lid check
// ---------------------------------------------------------------------------
template <typename T>
__global__ void pw_lid_kernel(const T *w, int nx, int ny, int nz, int nzp, int *flag) {
    int64_t n = (int64_t)nx * ny;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        int j = (int)(c % ny), i = (int)(c / ny);
        T x = w[((int64_t)(i + 2) * (ny + 4) + (j + 2)) * nzp + (nz - 1)];
        if (pw_to<float>(x) != 0.0f || pw_to<double>(x) != 0.0) atomicOr(flag, 1);
    }
}

extern "C" pw_status pw_check_lid(const pw_mesh *m, const void *w, void *stream) {
    if (!m) return pw_fail(PW_ERR_ARG, "mesh is NULL");
    pw_status s;
    if ((s = pw_check_ptr(w, "w")) != PW_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    int *d = m->status + 1;  // the mesh's lid flag word
    PW_CUDA(cudaMemsetAsync(d, 0, sizeof(int), st));
    if (m->dtype == PW_F64) pw_lid_kernel<double><<<m->num_sms * 2, 256, 0, st>>>((const double *)w, m->nx, m->ny, m->nz, m->nzp, d);
    else if (m->dtype == PW_F32) pw_lid_kernel<float><<<m->num_sms * 2, 256, 0, st>>>((const float *)w, m->nx, m->ny, m->nz, m->nzp, d);
    else pw_lid_kernel<__nv_bfloat16><<<m->num_sms * 2, 256, 0, st>>>((const __nv_bfloat16 *)w, m->nx, m->ny, m->nz, m->nzp, d);
    PW_CUDA(cudaGetLastError());
    int h = 0;
    PW_CUDA(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st));
    PW_CUDA(cudaStreamSynchronize(st));
    return h ? pw_fail(PW_ERR_LID, "w has non-zero values on the lid face k = nz-1") : PW_OK;
}
