// pw_static.cu -- the conservation sums without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need the
// diagnostics: a caching allocator (PyTorch's, or a model's own pool) may hold
// all free device memory, so a raw cudaMalloc fails or would fragment it, and
// inside a tight time-stepping loop an allocation can synchronise the device
// and stall the stream.  Such a caller may also have no mesh object, since
// creating one allocates.  pw_residuals_noalloc serves them: the caller passes
// the field/source buffers, the layout and the energy weights (host arrays),
// and the library uses a file-scope device array as its only scratch.
#include "pw_internal.h"

// Scratch: the reduction records (PW_RED_SCRATCH doubles: the block partials
// and the totals), then the two weight columns (PW_NOALLOC_MAX_NZ doubles each).
// Every GPU that loads the library holds this array (about 125 KB) until the
// process exits.
static __device__ __align__(256) double pw_noalloc_scratch[PW_RED_SCRATCH + 2 * PW_NOALLOC_MAX_NZ];

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress, with the device current.  It is looked up on every call
// (a cheap host query; the call synchronises its stream anyway): a context
// re-created after cudaDeviceReset may place the array elsewhere, so a cached
// address could go stale.
static pw_status pw_noalloc_scratch_ptr(double **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, pw_noalloc_scratch);
    if (e != cudaSuccess) return pw_cuda_fail(e, "cudaGetSymbolAddress(pw_noalloc_scratch)");
    if (!p) return pw_fail(PW_ERR_CUDA, "cudaGetSymbolAddress returned NULL");
    *out = (double *)p;
    return PW_OK;
}

// The fields must be device (or managed) memory of the current device: a host
// pointer or another GPU's buffer would otherwise reach the kernel and fault.
static pw_status pw_check_device_ptr(const void *p, const char *name, int dev) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of an unknown pointer
        return pw_fail(PW_ERR_ARG, "%s is not a CUDA allocation", name);
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return pw_fail(PW_ERR_ARG, "%s is not device memory (memory type %d)", name, (int)a.type);
    if (a.type == cudaMemoryTypeDevice && a.device != dev)
        return pw_fail(PW_ERR_ARG, "%s lives on device %d, the current device is %d", name, a.device, dev);
    return PW_OK;
}

extern "C" pw_status pw_residuals_noalloc(int nx, int ny, int nz, int nzp, pw_dtype dtype,
                                          const double *w_uv, const double *w_w, const void *u,
                                          const void *v, const void *w, const void *su, const void *sv,
                                          const void *sw, double *out, void *stream) {
    if (nx < 1 || ny < 1 || nz < 1)
        return pw_fail(PW_ERR_SHAPE, "bad sizes nx=%d ny=%d nz=%d", nx, ny, nz);
    if (nz > PW_NOALLOC_MAX_NZ)
        return pw_fail(PW_ERR_SHAPE, "nz=%d exceeds the no-allocation limit PW_NOALLOC_MAX_NZ=%d", nz,
                       PW_NOALLOC_MAX_NZ);
    if (nzp < nz || nzp % 8 != 0)
        return pw_fail(PW_ERR_SHAPE, "nzp=%d must be >= nz and a multiple of 8", nzp);
    if ((int64_t)(nx + 4) * (ny + 4) > (int64_t)1 << 31)
        return pw_fail(PW_ERR_SHAPE, "horizontal size too large");
    if (dtype != PW_F64 && dtype != PW_F32 && dtype != PW_BF16 && dtype != PW_BF16_OUT)
        return pw_fail(PW_ERR_DTYPE, "unknown dtype %d", (int)dtype);
    if (!w_uv || !w_w || !out) return pw_fail(PW_ERR_ARG, "w_uv, w_w and out must not be NULL");
    const void *ps[6] = {u, v, w, su, sv, sw};
    const char *nm[6] = {"u", "v", "w", "su", "sv", "sw"};
    int dev = 0;
    PW_CUDA(cudaGetDevice(&dev));
    for (int q = 0; q < 6; q++) {
        pw_status s = pw_check_ptr(ps[q], nm[q]);
        if (s == PW_OK) s = pw_check_device_ptr(ps[q], nm[q], dev);
        if (s != PW_OK) return s;
    }
    double *scratch = nullptr;
    pw_status s = pw_noalloc_scratch_ptr(&scratch);
    if (s != PW_OK) return s;
    // every entry of the reduction records is rewritten by each pass; the
    // finished-block counter (zero-initialised) is back at 0 after each
    double *wuv = scratch + PW_RED_SCRATCH, *ww = wuv + PW_NOALLOC_MAX_NZ;
    cudaStream_t st = (cudaStream_t)stream;
    PW_CUDA(cudaMemcpyAsync(wuv, w_uv, (size_t)nz * sizeof(double), cudaMemcpyHostToDevice, st));
    PW_CUDA(cudaMemcpyAsync(ww, w_w, (size_t)nz * sizeof(double), cudaMemcpyHostToDevice, st));
    s = pw_residuals_run(nx, ny, nz, nzp, dtype, wuv, ww, u, v, w, su, sv, sw, scratch, nullptr, out, st);
    if (s != PW_OK) return s;
    return PW_OK;
}
