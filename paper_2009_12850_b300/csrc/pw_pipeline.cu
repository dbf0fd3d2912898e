// pw_pipeline.cu -- the PW step on fields that live in host memory, with the
// host<->device copies overlapped with the device work slab by slab.
//
// The paper's hybrid code copies u, v, w to the GPU every timestep, advects on
// the device while the CPU runs its own dynamics, and copies the sources back;
// the copies are asynchronous, and the authors note that integrating the
// sources as they stream back would overlap the CPU's work with the copy
// (sections 3 and 3.1).  Here one call takes host arrays in the library layout
// and runs, on three streams:
//   copy-in   : interior rows of u, v, w (and of the old sources when beta = 1)
//               one x-slab at a time (2-D copies, so host halos are not read);
//   compute   : y halos of each arrived slab; the periodic x-halo columns -1 and
//               nx are device copies of columns nx-1 and 0 (column nx-1 is sent
//               first for that reason); the stencil of slab s runs once slab
//               s+1 has arrived (it reads one column beyond each slab edge);
//   copy-out  : interior rows of su, sv, sw of each finished slab, followed by
//               the caller's per-slab callback, if any.
// Only the columns -1 and nx of the x halo are filled: the stencils read one
// column beyond each edge.  Device copies of the six fields are owned by the
// pipeline object.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pw_internal.h"

struct pw_slab_note {
    pw_slab_fn fn;
    void *user;
    int i0, i1;
};

struct pw_pipeline {
    const pw_mesh *mesh;
    int slab, nslab;
    void *dev[6];  // u, v, w, su, sv, sw on the device (library layout)
    std::vector<void *> sdev;  // scalars then their sources (pw_pipeline_reserve_scalars)
    cudaStream_t s_in, s_c, s_out;
    cudaEvent_t ev_start, ev_last, ev_done;
    std::vector<cudaEvent_t> ev_in, ev_c;
    std::vector<pw_slab_note> notes;
    bool notes_pending;  // host callbacks of the previous call may still run
};

// y halos (rows -2, -1, ny, ny+1) of columns [i_begin, i_end) of up to three
// fields: one warp per (column, halo row), 16-byte copies of the used levels
__global__ void pw_yhalo_kernel(char *f0, char *f1, char *f2, int ny, int64_t col_stride, int nchunk,
                                int i_begin, int i_end) {
    char *f = blockIdx.y == 0 ? f0 : blockIdx.y == 1 ? f1 : f2;
    const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5);
    if (c >= 4LL * (i_end - i_begin)) return;
    const int ih = i_begin + 2 + (int)(c / 4), s = (int)(c % 4);
    const int jh = s < 2 ? s : ny + s;         // 0, 1, ny+2, ny+3
    const int js = s < 2 ? ny + s : s;         // the periodic image: ny, ny+1, 2, 3
    const int4 *src = reinterpret_cast<const int4 *>(f + ((int64_t)ih * (ny + 4) + js) * col_stride);
    int4 *dst = reinterpret_cast<int4 *>(f + ((int64_t)ih * (ny + 4) + jh) * col_stride);
    for (int q = lane; q < nchunk; q += 32) dst[q] = src[q];
}

// the fields of one host step: device and host base pointers, element size
struct pw_field_pair {
    char *dev, *host;
    size_t es;
};

// y halos of columns [i_begin, i_end) of the input fields, three per launch
static pw_status pw_yhalo(const pw_pipeline *p, const std::vector<pw_field_pair> &in, int i_begin, int i_end) {
    const pw_mesh *m = p->mesh;
    const int es = pw_elem_in(m->dtype);
    const int64_t col_stride = (int64_t)m->nzp * es;
    const int nchunk = (int)(((int64_t)m->nz * es + 15) / 16);
    const int64_t work = 4LL * (i_end - i_begin);
    const int warps = 8;
    for (size_t f = 0; f < in.size(); f += 3) {
        const int nf = (int)std::min<size_t>(3, in.size() - f);
        char *f0 = in[f].dev, *f1 = nf > 1 ? in[f + 1].dev : f0, *f2 = nf > 2 ? in[f + 2].dev : f0;
        dim3 grid((unsigned)((work + warps - 1) / warps), (unsigned)nf);
        pw_yhalo_kernel<<<grid, warps * 32, 0, p->s_c>>>(f0, f1, f2, m->ny, col_stride, nchunk, i_begin, i_end);
        PW_CUDA(cudaGetLastError());
    }
    return PW_OK;
}

// whole column (halo rows included) src -> dst of the input fields, in halo column indices
static pw_status pw_copy_column(const pw_pipeline *p, const std::vector<pw_field_pair> &in, int dst_col,
                                int src_col) {
    const size_t col = (size_t)p->mesh->si * (size_t)pw_elem_in(p->mesh->dtype);
    for (const pw_field_pair &f : in)
        PW_CUDA(cudaMemcpyAsync(f.dev + (size_t)dst_col * col, f.dev + (size_t)src_col * col, col,
                                cudaMemcpyDeviceToDevice, p->s_c));
    return PW_OK;
}

// interior points (levels k < nz of rows j in [0, ny)) of columns [i0, i1) of the
// listed fields between host and device: one 2-D copy per field when columns
// have no padding levels, else a 3-D copy that leaves the padding alone
static pw_status pw_copy_rows(const pw_pipeline *p, const std::vector<pw_field_pair> &fields, int i0, int i1,
                              bool to_device, cudaStream_t st) {
    if (i1 <= i0) return PW_OK;
    const pw_mesh *m = p->mesh;
    const cudaMemcpyKind kind = to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
    for (const pw_field_pair &f : fields) {
        const size_t pitch = (size_t)m->si * f.es;
        const size_t off = (size_t)(i0 + 2) * pitch + 2 * (size_t)m->sj * f.es;
        char *dst = to_device ? f.dev : f.host;
        char *src = to_device ? f.host : f.dev;
        if (m->nzp == m->nz) {
            const size_t width = (size_t)m->ny * (size_t)m->sj * f.es;
            PW_CUDA(cudaMemcpy2DAsync(dst + off, pitch, src + off, pitch, width, (size_t)(i1 - i0), kind, st));
        } else {
            // rows of nz levels, row pitch nzp levels, ny + 4 rows per column
            cudaMemcpy3DParms c = {};
            const size_t row = (size_t)m->nzp * f.es;
            c.srcPtr = make_cudaPitchedPtr(src + off, row, (size_t)m->nz * f.es, (size_t)m->ny + 4);
            c.dstPtr = make_cudaPitchedPtr(dst + off, row, (size_t)m->nz * f.es, (size_t)m->ny + 4);
            c.extent = make_cudaExtent((size_t)m->nz * f.es, (size_t)m->ny, (size_t)(i1 - i0));
            c.kind = kind;
            PW_CUDA(cudaMemcpy3DAsync(&c, st));
        }
    }
    return PW_OK;
}

// the stencils on columns [i0, i1): a view of the mesh that starts at column i0
// (in: u, v, w, scalars; out: su, sv, sw, scalar sources)
static pw_status pw_slab_advect(const pw_pipeline *p, const std::vector<pw_field_pair> &in,
                                const std::vector<pw_field_pair> &out, int i0, int i1, int beta) {
    const pw_mesh *m = p->mesh;
    pw_mesh view = *m;
    view.nx = i1 - i0;
    const size_t ei = (size_t)pw_elem_in(m->dtype) * (size_t)m->si * (size_t)i0;
    const size_t eo = (size_t)pw_elem_out(m->dtype) * (size_t)m->si * (size_t)i0;
    pw_status s = pw_launch_advect(&view, in[0].dev + ei, in[1].dev + ei, in[2].dev + ei, out[0].dev + eo,
                                   out[1].dev + eo, out[2].dev + eo, beta, p->s_c, m->tile_j, m->tile_i);
    const int n = (int)in.size() - 3;
    if (s != PW_OK || n == 0) return s;
    const void *phi[PW_MAX_SCALARS];
    void *sphi[PW_MAX_SCALARS];
    for (int a = 0; a < n; a++) {
        phi[a] = in[3 + a].dev + ei;
        sphi[a] = out[3 + a].dev + eo;
    }
    return pw_launch_advect_scalars(&view, in[0].dev + ei, in[1].dev + ei, in[2].dev + ei, n, phi, sphi, beta,
                                    p->s_c, m->tile_j, m->tile_i, 0);
}

static void CUDART_CB pw_slab_note_fn(void *arg) {
    const pw_slab_note *n = (const pw_slab_note *)arg;
    n->fn(n->user, n->i0, n->i1);
}

extern "C" void pw_pipeline_destroy(pw_pipeline *p) {
    if (!p) return;
    if (p->s_c) cudaStreamSynchronize(p->s_c);
    if (p->s_in) cudaStreamSynchronize(p->s_in);
    if (p->s_out) cudaStreamSynchronize(p->s_out);
    for (int f = 0; f < 6; f++) cudaFree(p->dev[f]);
    for (void *d : p->sdev) cudaFree(d);
    for (cudaEvent_t e : p->ev_in) cudaEventDestroy(e);
    for (cudaEvent_t e : p->ev_c) cudaEventDestroy(e);
    if (p->ev_start) cudaEventDestroy(p->ev_start);
    if (p->ev_last) cudaEventDestroy(p->ev_last);
    if (p->ev_done) cudaEventDestroy(p->ev_done);
    if (p->s_in) cudaStreamDestroy(p->s_in);
    if (p->s_c) cudaStreamDestroy(p->s_c);
    if (p->s_out) cudaStreamDestroy(p->s_out);
    delete p;
}

extern "C" pw_status pw_pipeline_create(const pw_mesh *m, int slab, pw_pipeline **out) {
    if (!m || !out) return pw_fail(PW_ERR_ARG, "mesh and out must not be NULL");
    *out = nullptr;
    if (slab < 0) return pw_fail(PW_ERR_ARG, "slab = %d columns (>= 0)", slab);
    if (slab == 0) slab = std::max(1, (m->nx + 31) / 32);
    slab = std::min(slab, m->nx);
    pw_pipeline *p = new (std::nothrow) pw_pipeline();
    if (!p) return pw_fail(PW_ERR_NOMEM, "pipeline object");
    p->mesh = m;
    p->slab = slab;
    p->nslab = (m->nx + slab - 1) / slab;
    p->notes_pending = false;
    cudaError_t e = cudaSuccess;
    do {
        for (int f = 0; f < 6 && e == cudaSuccess; f++) {
            const size_t es = (size_t)(f < 3 ? pw_elem_in(m->dtype) : pw_elem_out(m->dtype));
            e = cudaMalloc(&p->dev[f], (size_t)m->total * es);
            if (e == cudaSuccess) e = cudaMemset(p->dev[f], 0, (size_t)m->total * es);
        }
        if (e != cudaSuccess) break;
        if ((e = cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaStreamCreateWithFlags(&p->s_c, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming)) != cudaSuccess) break;
        if ((e = cudaEventCreateWithFlags(&p->ev_last, cudaEventDisableTiming)) != cudaSuccess) break;
        if ((e = cudaEventCreateWithFlags(&p->ev_done, cudaEventDisableTiming)) != cudaSuccess) break;
        p->ev_in.assign(p->nslab, nullptr);
        p->ev_c.assign(p->nslab, nullptr);
        for (int s = 0; s < p->nslab && e == cudaSuccess; s++) {
            e = cudaEventCreateWithFlags(&p->ev_in[s], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_c[s], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) break;
        e = cudaDeviceSynchronize();  // the zeroed buffers are ready before any stream uses them
    } while (0);
    if (e != cudaSuccess) {
        pw_pipeline_destroy(p);
        return pw_cuda_fail(e, "pipeline set-up");
    }
    p->notes.resize(p->nslab);
    *out = p;
    return PW_OK;
}

extern "C" pw_status pw_pipeline_slab(const pw_pipeline *p, int *slab, int *nslab) {
    if (!p) return pw_fail(PW_ERR_ARG, "pipeline is NULL");
    if (slab) *slab = p->slab;
    if (nslab) *nslab = p->nslab;
    return PW_OK;
}

extern "C" pw_status pw_pipeline_sync(pw_pipeline *p) {
    if (!p) return pw_fail(PW_ERR_ARG, "pipeline is NULL");
    PW_CUDA(cudaEventSynchronize(p->ev_done));
    p->notes_pending = false;
    return PW_OK;
}

extern "C" pw_status pw_pipeline_reserve_scalars(pw_pipeline *p, int n) {
    if (!p) return pw_fail(PW_ERR_ARG, "pipeline is NULL");
    if (n < 0 || n > PW_MAX_SCALARS) return pw_fail(PW_ERR_ARG, "n = %d scalars (0..%d)", n, PW_MAX_SCALARS);
    const int have = (int)p->sdev.size() / 2;
    if (n <= have) return PW_OK;
    const pw_mesh *m = p->mesh;
    PW_CUDA(cudaDeviceSynchronize());  // no step of this pipeline is in flight while buffers change
    std::vector<void *> fresh(2 * (size_t)n, nullptr);
    cudaError_t e = cudaSuccess;
    for (int a = 0; a < 2 * n && e == cudaSuccess; a++) {
        const bool src = a >= n;
        const int q = src ? a - n : a;
        if (q < have) {  // keep the buffers already there
            fresh[a] = p->sdev[(src ? have : 0) + q];
            continue;
        }
        const size_t bytes = (size_t)m->total * (size_t)(src ? pw_elem_out(m->dtype) : pw_elem_in(m->dtype));
        e = cudaMalloc(&fresh[a], bytes);
        if (e == cudaSuccess) e = cudaMemset(fresh[a], 0, bytes);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        for (int a = 0; a < 2 * n; a++) {
            const bool src = a >= n;
            const int q = src ? a - n : a;
            if (q >= have) cudaFree(fresh[a]);
        }
        return pw_cuda_fail(e, "pipeline scalar buffers");
    }
    p->sdev.swap(fresh);
    return PW_OK;
}

// The step on host arrays: the wind and n scalars in, their sources out.
static pw_status pw_host_step(pw_pipeline *p, const void *const *host_in, void *const *host_out, int n,
                              int beta, pw_slab_fn on_slab, void *user, cudaStream_t user_st) {
    const pw_mesh *m = p->mesh;
    const int have = (int)p->sdev.size() / 2;
    if (n > have)
        return pw_fail(PW_ERR_ARG, "%d scalars but buffers for %d reserved (pw_pipeline_reserve_scalars)", n, have);
    std::vector<pw_field_pair> in, out;
    const size_t ei = (size_t)pw_elem_in(m->dtype), eo = (size_t)pw_elem_out(m->dtype);
    for (int f = 0; f < 3 + n; f++) {
        char *din = (char *)(f < 3 ? p->dev[f] : p->sdev[f - 3]);
        char *dout = (char *)(f < 3 ? p->dev[3 + f] : p->sdev[have + f - 3]);
        in.push_back(pw_field_pair{din, (char *)host_in[f], ei});
        out.push_back(pw_field_pair{dout, (char *)host_out[f], eo});
    }
    // the notes of the previous call are read by its callbacks: let them finish
    if (p->notes_pending) {
        PW_CUDA(cudaEventSynchronize(p->ev_done));
        p->notes_pending = false;
    }
    const int last = m->nx - 1;
    const bool precopy = p->nslab > 1;
    pw_status st;

    PW_CUDA(cudaEventRecord(p->ev_start, user_st));
    PW_CUDA(cudaStreamWaitEvent(p->s_in, p->ev_start, 0));
    PW_CUDA(cudaStreamWaitEvent(p->s_c, p->ev_start, 0));
    PW_CUDA(cudaStreamWaitEvent(p->s_out, p->ev_start, 0));

    // copy-in: column nx-1 first (the x halo of slab 0), then the slabs in order;
    // with beta = 1 the old sources travel too
    if (precopy) {
        if ((st = pw_copy_rows(p, in, last, last + 1, true, p->s_in)) != PW_OK) return st;
        PW_CUDA(cudaEventRecord(p->ev_last, p->s_in));
    }
    for (int s = 0; s < p->nslab; s++) {
        const int i0 = s * p->slab, i1 = std::min(m->nx, i0 + p->slab);
        const int i1w = (precopy && s == p->nslab - 1) ? std::min(i1, last) : i1;  // nx-1 already there
        if ((st = pw_copy_rows(p, in, i0, i1w, true, p->s_in)) != PW_OK) return st;
        if (beta && (st = pw_copy_rows(p, out, i0, i1, true, p->s_in)) != PW_OK) return st;
        PW_CUDA(cudaEventRecord(p->ev_in[s], p->s_in));
    }

    // compute: halos as the slabs arrive, the stencils one slab behind
    if (precopy) {
        PW_CUDA(cudaStreamWaitEvent(p->s_c, p->ev_last, 0));
        if ((st = pw_yhalo(p, in, last, last + 1)) != PW_OK) return st;
        if ((st = pw_copy_column(p, in, 1, last + 2)) != PW_OK) return st;  // column -1 <- nx-1
    }
    for (int s = 0; s < p->nslab; s++) {
        const int i0 = s * p->slab, i1 = std::min(m->nx, i0 + p->slab);
        PW_CUDA(cudaStreamWaitEvent(p->s_c, p->ev_in[s], 0));
        if ((st = pw_yhalo(p, in, i0, i1)) != PW_OK) return st;
        if (s == 0) {
            if (!precopy && (st = pw_copy_column(p, in, 1, last + 2)) != PW_OK) return st;
            if ((st = pw_copy_column(p, in, m->nx + 2, 2)) != PW_OK) return st;  // column nx <- 0
        }
        if (s >= 1) {
            const int j0 = (s - 1) * p->slab;
            if ((st = pw_slab_advect(p, in, out, j0, i0, beta)) != PW_OK) return st;
            PW_CUDA(cudaEventRecord(p->ev_c[s - 1], p->s_c));
        }
    }
    {
        const int i0 = (p->nslab - 1) * p->slab;
        if ((st = pw_slab_advect(p, in, out, i0, m->nx, beta)) != PW_OK) return st;
        PW_CUDA(cudaEventRecord(p->ev_c[p->nslab - 1], p->s_c));
    }

    // copy-out, slab by slab, each followed by the caller's callback
    for (int s = 0; s < p->nslab; s++) {
        const int i0 = s * p->slab, i1 = std::min(m->nx, i0 + p->slab);
        PW_CUDA(cudaStreamWaitEvent(p->s_out, p->ev_c[s], 0));
        if ((st = pw_copy_rows(p, out, i0, i1, false, p->s_out)) != PW_OK) return st;
        if (on_slab) {
            p->notes[s] = pw_slab_note{on_slab, user, i0, i1};
            PW_CUDA(cudaLaunchHostFunc(p->s_out, pw_slab_note_fn, &p->notes[s]));
        }
    }
    PW_CUDA(cudaEventRecord(p->ev_done, p->s_out));
    PW_CUDA(cudaStreamWaitEvent(user_st, p->ev_done, 0));
    p->notes_pending = on_slab != nullptr;
    return PW_OK;
}

// pointers of one call: none NULL, no output aliasing an input or another output
static pw_status pw_check_host_fields(const void *const *in, void *const *out, int nf) {
    for (int f = 0; f < nf; f++) {
        if (!in[f]) return pw_fail(PW_ERR_ARG, "host input %d is NULL", f);
        if (!out[f]) return pw_fail(PW_ERR_ARG, "host output %d is NULL", f);
    }
    for (int a = 0; a < nf; a++)
        for (int b = 0; b < nf; b++) {
            if (out[a] == in[b]) return pw_fail(PW_ERR_ARG, "host output %d aliases input %d", a, b);
            if (b > a && out[a] == out[b]) return pw_fail(PW_ERR_ARG, "host outputs %d and %d alias", a, b);
        }
    return PW_OK;
}

extern "C" pw_status pw_advect_host(pw_pipeline *p, const void *u, const void *v, const void *w, void *su,
                                    void *sv, void *sw, int beta, pw_slab_fn on_slab, void *user, void *stream) {
    if (!p) return pw_fail(PW_ERR_ARG, "pipeline is NULL");
    if (beta != 0 && beta != 1) return pw_fail(PW_ERR_ARG, "beta must be 0 or 1");
    const void *in[3] = {u, v, w};
    void *out[3] = {su, sv, sw};
    pw_status s = pw_check_host_fields(in, out, 3);
    if (s != PW_OK) return s;
    return pw_host_step(p, in, out, 0, beta, on_slab, user, (cudaStream_t)stream);
}

extern "C" pw_status pw_advect_host_scalars(pw_pipeline *p, const void *u, const void *v, const void *w,
                                            void *su, void *sv, void *sw, int n, const void *const *phi,
                                            void *const *sphi, int beta, pw_slab_fn on_slab, void *user,
                                            void *stream) {
    if (!p) return pw_fail(PW_ERR_ARG, "pipeline is NULL");
    if (beta != 0 && beta != 1) return pw_fail(PW_ERR_ARG, "beta must be 0 or 1");
    if (n < 0 || n > PW_MAX_SCALARS) return pw_fail(PW_ERR_ARG, "n = %d scalars (0..%d)", n, PW_MAX_SCALARS);
    if (n > 0 && (!phi || !sphi)) return pw_fail(PW_ERR_ARG, "scalar pointer arrays are NULL");
    const void *in[3 + PW_MAX_SCALARS] = {u, v, w};
    void *out[3 + PW_MAX_SCALARS] = {su, sv, sw};
    for (int a = 0; a < n; a++) {
        in[3 + a] = phi[a];
        out[3 + a] = sphi[a];
    }
    pw_status s = pw_check_host_fields(in, out, 3 + n);
    if (s != PW_OK) return s;
    return pw_host_step(p, in, out, n, beta, on_slab, user, (cudaStream_t)stream);
}

extern "C" pw_status pw_pipeline_device_fields(const pw_pipeline *p, void **fields6) {
    if (!p || !fields6) return pw_fail(PW_ERR_ARG, "pipeline and fields6 must not be NULL");
    for (int f = 0; f < 6; f++) fields6[f] = p->dev[f];
    return PW_OK;
}
