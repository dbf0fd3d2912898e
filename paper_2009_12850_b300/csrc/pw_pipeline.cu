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

static pw_status pw_yhalo(const pw_pipeline *p, int i_begin, int i_end) {
    const pw_mesh *m = p->mesh;
    const int es = pw_elem_in(m->dtype);
    const int64_t col_stride = (int64_t)m->nzp * es;
    const int nchunk = (int)(((int64_t)m->nz * es + 15) / 16);
    const int64_t work = 4LL * (i_end - i_begin);
    const int warps = 8;
    dim3 grid((unsigned)((work + warps - 1) / warps), 3);
    pw_yhalo_kernel<<<grid, warps * 32, 0, p->s_c>>>((char *)p->dev[0], (char *)p->dev[1], (char *)p->dev[2],
                                                     m->ny, col_stride, nchunk, i_begin, i_end);
    PW_CUDA(cudaGetLastError());
    return PW_OK;
}

// whole column (halo rows included) src -> dst of u, v, w, in halo column indices
static pw_status pw_copy_column(const pw_pipeline *p, int dst_col, int src_col) {
    const pw_mesh *m = p->mesh;
    const size_t es = (size_t)pw_elem_in(m->dtype), col = (size_t)m->si * es;
    for (int f = 0; f < 3; f++) {
        char *b = (char *)p->dev[f];
        PW_CUDA(cudaMemcpyAsync(b + (size_t)dst_col * col, b + (size_t)src_col * col, col,
                                cudaMemcpyDeviceToDevice, p->s_c));
    }
    return PW_OK;
}

// interior rows of columns [i0, i1) of the fields [f_begin, f_end) between the
// host arrays and the device copies
static pw_status pw_copy_rows(const pw_pipeline *p, void *const *host, int f_begin, int f_end, int i0, int i1,
                              bool to_device, cudaStream_t st) {
    if (i1 <= i0) return PW_OK;
    const pw_mesh *m = p->mesh;
    for (int f = f_begin; f < f_end; f++) {
        const size_t es = (size_t)(f < 3 ? pw_elem_in(m->dtype) : pw_elem_out(m->dtype));
        const size_t pitch = (size_t)m->si * es;
        const size_t off = (size_t)(i0 + 2) * pitch + 2 * (size_t)m->sj * es;
        const size_t width = (size_t)m->ny * (size_t)m->sj * es;
        char *d = (char *)p->dev[f] + off;
        char *h = (char *)host[f] + off;
        if (to_device)
            PW_CUDA(cudaMemcpy2DAsync(d, pitch, h, pitch, width, (size_t)(i1 - i0), cudaMemcpyHostToDevice, st));
        else
            PW_CUDA(cudaMemcpy2DAsync(h, pitch, d, pitch, width, (size_t)(i1 - i0), cudaMemcpyDeviceToHost, st));
    }
    return PW_OK;
}

// the stencil on columns [i0, i1): a view of the mesh that starts at column i0
static pw_status pw_slab_advect(const pw_pipeline *p, int i0, int i1, int beta) {
    const pw_mesh *m = p->mesh;
    pw_mesh view = *m;
    view.nx = i1 - i0;
    const size_t ei = (size_t)pw_elem_in(m->dtype) * (size_t)m->si * (size_t)i0;
    const size_t eo = (size_t)pw_elem_out(m->dtype) * (size_t)m->si * (size_t)i0;
    return pw_launch_advect(&view, (char *)p->dev[0] + ei, (char *)p->dev[1] + ei, (char *)p->dev[2] + ei,
                            (char *)p->dev[3] + eo, (char *)p->dev[4] + eo, (char *)p->dev[5] + eo, beta, p->s_c,
                            m->tile_j, m->tile_i);
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

extern "C" pw_status pw_advect_host(pw_pipeline *p, const void *u, const void *v, const void *w, void *su,
                                    void *sv, void *sw, int beta, pw_slab_fn on_slab, void *user, void *stream) {
    if (!p) return pw_fail(PW_ERR_ARG, "pipeline is NULL");
    if (beta != 0 && beta != 1) return pw_fail(PW_ERR_ARG, "beta must be 0 or 1");
    void *host[6] = {(void *)u, (void *)v, (void *)w, su, sv, sw};
    const char *nm[6] = {"u", "v", "w", "su", "sv", "sw"};
    for (int f = 0; f < 6; f++)
        if (!host[f]) return pw_fail(PW_ERR_ARG, "host array %s is NULL", nm[f]);
    for (int a = 0; a < 3; a++)
        for (int b = 3; b < 6; b++)
            if (host[a] == host[b]) return pw_fail(PW_ERR_ARG, "%s and %s alias", nm[a], nm[b]);
    if (su == sv || su == sw || sv == sw) return pw_fail(PW_ERR_ARG, "outputs alias");
    const pw_mesh *m = p->mesh;
    cudaStream_t user_st = (cudaStream_t)stream;
    // the notes of the previous call are read by its callbacks: let them finish
    if (p->notes_pending) {
        PW_CUDA(cudaEventSynchronize(p->ev_done));
        p->notes_pending = false;
    }
    const int nf_in = beta ? 6 : 3;  // with beta = 1 the old sources travel too
    const int last = m->nx - 1;
    const bool precopy = p->nslab > 1;
    pw_status st;

    PW_CUDA(cudaEventRecord(p->ev_start, user_st));
    PW_CUDA(cudaStreamWaitEvent(p->s_in, p->ev_start, 0));
    PW_CUDA(cudaStreamWaitEvent(p->s_c, p->ev_start, 0));
    PW_CUDA(cudaStreamWaitEvent(p->s_out, p->ev_start, 0));

    // copy-in: column nx-1 first (the x halo of slab 0), then the slabs in order
    if (precopy) {
        if ((st = pw_copy_rows(p, host, 0, 3, last, last + 1, true, p->s_in)) != PW_OK) return st;
        PW_CUDA(cudaEventRecord(p->ev_last, p->s_in));
    }
    for (int s = 0; s < p->nslab; s++) {
        const int i0 = s * p->slab, i1 = std::min(m->nx, i0 + p->slab);
        const int i1w = (precopy && s == p->nslab - 1) ? std::min(i1, last) : i1;  // nx-1 already there
        if ((st = pw_copy_rows(p, host, 0, 3, i0, i1w, true, p->s_in)) != PW_OK) return st;
        if (beta && (st = pw_copy_rows(p, host, 3, nf_in, i0, i1, true, p->s_in)) != PW_OK) return st;
        PW_CUDA(cudaEventRecord(p->ev_in[s], p->s_in));
    }

    // compute: halos as the slabs arrive, the stencil one slab behind
    if (precopy) {
        PW_CUDA(cudaStreamWaitEvent(p->s_c, p->ev_last, 0));
        if ((st = pw_yhalo(p, last, last + 1)) != PW_OK) return st;
        if ((st = pw_copy_column(p, 1, last + 2)) != PW_OK) return st;  // column -1 <- nx-1
    }
    for (int s = 0; s < p->nslab; s++) {
        const int i0 = s * p->slab, i1 = std::min(m->nx, i0 + p->slab);
        PW_CUDA(cudaStreamWaitEvent(p->s_c, p->ev_in[s], 0));
        if ((st = pw_yhalo(p, i0, i1)) != PW_OK) return st;
        if (s == 0) {
            if (!precopy && (st = pw_copy_column(p, 1, last + 2)) != PW_OK) return st;
            if ((st = pw_copy_column(p, m->nx + 2, 2)) != PW_OK) return st;  // column nx <- 0
        }
        if (s >= 1) {
            const int j0 = (s - 1) * p->slab;
            if ((st = pw_slab_advect(p, j0, i0, beta)) != PW_OK) return st;
            PW_CUDA(cudaEventRecord(p->ev_c[s - 1], p->s_c));
        }
    }
    {
        const int i0 = (p->nslab - 1) * p->slab;
        if ((st = pw_slab_advect(p, i0, m->nx, beta)) != PW_OK) return st;
        PW_CUDA(cudaEventRecord(p->ev_c[p->nslab - 1], p->s_c));
    }

    // copy-out, slab by slab, each followed by the caller's callback
    for (int s = 0; s < p->nslab; s++) {
        const int i0 = s * p->slab, i1 = std::min(m->nx, i0 + p->slab);
        PW_CUDA(cudaStreamWaitEvent(p->s_out, p->ev_c[s], 0));
        if ((st = pw_copy_rows(p, host, 3, 6, i0, i1, false, p->s_out)) != PW_OK) return st;
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

extern "C" pw_status pw_pipeline_device_fields(const pw_pipeline *p, void **fields6) {
    if (!p || !fields6) return pw_fail(PW_ERR_ARG, "pipeline and fields6 must not be NULL");
    for (int f = 0; f < 6; f++) fields6[f] = p->dev[f];
    return PW_OK;
}
