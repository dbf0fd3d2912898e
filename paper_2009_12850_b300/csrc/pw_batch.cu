// pw_batch.cu -- batched ensembles (many uneven subdomains in one persistent
// launch) and the tile autotuner.
//
// A batch holds n FP32 meshes.  Each member is cut into x-march tiles whose
// shape depends on its column length (size class): with T threads per CTA and
// nkt = kc/4 threads per column, a tile has tile_j = T / nkt rows.  All tiles
// of all members are numbered in one flat list, members with the most work per
// tile first; CTAs (number of SMs x resident CTAs) pull tile numbers from a
// device counter and run the same x-march as the single-mesh kernel, with the
// member's TMA descriptors read from global memory.  The counter is reset by a
// memset node on the launch stream, so the whole step can be graph-captured.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "pw_march.cuh"

struct __align__(128) PwBatchMember {
    CUtensorMap maps[3];   // u, v, w (64-byte aligned, read by TMA from global memory)
    PwGeom g;
    float *su, *sv, *sw;
    const float *coef;
    int tiles_j, tiles_i, tiles_k, first_tile;
    int halo_first;        // first halo column (x3 fields) of this member in the halo launch
    int pad_[3];
};

struct pw_batch_impl {
    int n;
    std::vector<pw_mesh *> meshes;
    std::vector<PwBatchMember> host;   // in work order
    std::vector<int> order;            // member index of each slot
    PwBatchMember *dev = nullptr;
    int *counter = nullptr;
    int *status = nullptr;
    std::vector<void *> ptr[6];        // bound u v w su sv sw (by member index)
    bool bound = false;
    int threads = 256, tile_i = 32;
    int persistent = 1;                // 1: SMs x occupancy CTAs pull tiles; 0: one CTA per tile
    int grid = 0, total_tiles = 0, halo_cols = 0;
    size_t smem = 0;
};

struct pw_batch {
    pw_batch_impl impl;
};

static constexpr int PW_BATCH_NS = PW_MARCH_NS;

// persistent = 1: CTAs pull tile numbers from the counter until none is left;
// persistent = 0: CTA b runs tile b (the hardware block scheduler hands out the
// tiles in the same longest-first order)
__global__ void __launch_bounds__(512)
pw_batch_kernel(const PwBatchMember *__restrict__ members, int n, int total_tiles,
                int *__restrict__ counter, int *__restrict__ status, int beta, int persistent) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_tile;
    for (int pass = 0;; pass++) {
        int t;
        if (persistent) {
            if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1);
            __syncthreads();
            t = s_tile;
            __syncthreads();
        } else {
            if (pass > 0) return;
            t = blockIdx.x;
        }
        if (t >= total_tiles || pw_cta_failed(status)) return;
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (members[mid].first_tile <= t) lo = mid;
            else hi = mid - 1;
        }
        const PwBatchMember &M = members[lo];
        const PwGeom g = M.g;
        int local = t - M.first_tile;
        const int tjx = local % M.tiles_j;
        local /= M.tiles_j;
        const int tix = local % M.tiles_i, tkx = local / M.tiles_i;
        if (!pw_march_tile<float, float, float, 4, PW_MARCH_NS>(&M.maps[0], &M.maps[1], &M.maps[2], M.su, M.sv,
                                                   M.sw, M.coef, g, beta, status, smem_raw,
                                                   tjx * g.tj, tix * g.ti, tkx * g.kc))
            return;
    }
}

// periodic halo fill of the bound u, v, w of every member: one warp per halo
// column (same column mapping as the single-mesh halo kernel)
__global__ void pw_batch_halo_kernel(const PwBatchMember *__restrict__ members, int n, int total_cols,
                                     const void *const *__restrict__ fields) {
    const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * warps + (threadIdx.x >> 5);
    if (c >= total_cols) return;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (members[mid].halo_first <= c) lo = mid;
        else hi = mid - 1;
    }
    const PwGeom &g = members[lo].g;
    const int nx = g.nx, ny = g.ny;
    const int per_field = 4 * (ny + 4) + 4 * nx;
    int local = c - members[lo].halo_first;
    const int f = local / per_field;
    local -= f * per_field;
    char *base = (char *)fields[3 * lo + f];
    int ih, jh;
    if (local < 4 * (ny + 4)) {
        const int r = local / (ny + 4);
        ih = r < 2 ? r : nx + r;
        jh = local % (ny + 4);
    } else {
        const int q = local - 4 * (ny + 4);
        ih = 2 + q / 4;
        const int s = q % 4;
        jh = s < 2 ? s : ny + s;
    }
    const int is = ((ih - 2) % nx + nx) % nx + 2, js = ((jh - 2) % ny + ny) % ny + 2;
    const long long col = (long long)g.nzp * 4;
    const int4 *src = reinterpret_cast<const int4 *>(base + ((long long)is * (ny + 4) + js) * col);
    int4 *dst = reinterpret_cast<int4 *>(base + ((long long)ih * (ny + 4) + jh) * col);
    const int nchunk = (g.nz * 4 + 15) / 16;
    for (int q = lane; q < nchunk; q += 32) dst[q] = src[q];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PwGeom pw_member_geom(const pw_mesh *m, int threads, int tile_i) {
    PwGeom g;
    g.nx = m->nx;
    g.ny = m->ny;
    g.nz = m->nz;
    g.nzp = m->nzp;
    g.h = 4;
    const int kc_one = (m->nz + 3) / 4 * 4;
    g.kc = (kc_one + 8 <= 256) ? kc_one : 128;
    g.kb = g.kc + 8;
    const int nkt = g.kc / 4;
    g.tj = std::max(1, std::min(32, threads / nkt));
    g.ti = tile_i;
    g.ns = PW_BATCH_NS;
    g.plane_elems = (g.tj + 2) * g.kb;
    g.field_stride = (g.plane_elems + 31) / 32 * 32;
    g.si = m->si;
    g.sj = m->sj;
    g.tcx = m->tcx;
    g.tcy = m->tcy;
    g.ftcx = (float)m->tcx;
    g.ftcy = (float)m->tcy;
    return g;
}

static size_t pw_member_smem(const PwGeom &g) {
    return (size_t)g.ns * 3 * g.field_stride * sizeof(float) + (size_t)g.ns * sizeof(uint64_t);
}

// device array of the 3n bound field pointers used by the batched halo fill
static void **pw_batch_field_table(pw_batch_impl &b) {
    return reinterpret_cast<void **>(reinterpret_cast<char *>(b.status) + 64);
}

// (re)build member descriptors for the current tile configuration and upload
static pw_status pw_batch_build(pw_batch_impl &b, cudaStream_t st) {
    const int n = b.n;
    std::vector<PwGeom> geo(n);
    std::vector<double> work(n);
    for (int q = 0; q < n; q++) {
        geo[q] = pw_member_geom(b.meshes[q], b.threads, b.tile_i);
        if ((geo[q].kc / 4) > b.threads)
            return pw_fail(PW_ERR_SHAPE, "member %d needs at least %d threads per CTA", q, geo[q].kc / 4);
        work[q] = (double)geo[q].tj * geo[q].ti * geo[q].kc;
    }
    b.order.resize(n);
    for (int q = 0; q < n; q++) b.order[q] = q;
    std::stable_sort(b.order.begin(), b.order.end(), [&](int a, int c) { return work[a] > work[c]; });
    b.host.assign(n, PwBatchMember{});
    int first = 0, halo = 0;
    size_t smem = 0;
    for (int s = 0; s < n; s++) {
        const int q = b.order[s];
        const pw_mesh *m = b.meshes[q];
        PwBatchMember &M = b.host[s];
        M.g = geo[q];
        M.tiles_j = (m->ny + M.g.tj - 1) / M.g.tj;
        M.tiles_i = (m->nx + M.g.ti - 1) / M.g.ti;
        M.tiles_k = (m->nz + M.g.kc - 1) / M.g.kc;
        M.first_tile = first;
        first += M.tiles_j * M.tiles_i * M.tiles_k;
        M.halo_first = halo;
        halo += 3 * (4 * (m->ny + 4) + 4 * m->nx);
        M.coef = m->coef32;
        smem = std::max(smem, pw_member_smem(M.g));
        if (b.bound) {
            M.su = (float *)b.ptr[3][q];
            M.sv = (float *)b.ptr[4][q];
            M.sw = (float *)b.ptr[5][q];
            for (int f = 0; f < 3; f++) {
                pw_status s2 = pw_make_field_map(&M.maps[f], b.ptr[f][q], PW_F32, m->nx, m->ny, m->nzp,
                                                 pw_kdim(m->nz, f), M.g.kb, M.g.tj + 2);
                if (s2 != PW_OK) return s2;
            }
        }
    }
    if (smem > 226 * 1024) return pw_fail(PW_ERR_SHAPE, "batch tile needs %zu bytes of shared memory", smem);
    b.total_tiles = first;
    b.halo_cols = halo;
    b.smem = smem;
    PW_CUDA(cudaFuncSetAttribute(pw_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pw_batch_kernel, b.threads, smem));
    if (per_sm < 1) return pw_fail(PW_ERR_SHAPE, "batch kernel cannot be resident with %d threads", b.threads);
    b.grid = b.persistent ? std::min(b.total_tiles, per_sm * b.meshes[0]->num_sms) : b.total_tiles;
    PW_CUDA(cudaMemcpyAsync(b.dev, b.host.data(), sizeof(PwBatchMember) * n, cudaMemcpyHostToDevice, st));
    if (b.bound) {
        // the halo launch addresses members by slot: its field table must follow
        // the work order of this build, which changes with the tile shape
        std::vector<void *> tab(3 * (size_t)n);
        for (int slot = 0; slot < n; slot++)
            for (int f = 0; f < 3; f++) tab[3 * slot + f] = b.ptr[f][b.order[slot]];
        PW_CUDA(cudaMemcpyAsync(pw_batch_field_table(b), tab.data(), sizeof(void *) * 3 * n,
                                cudaMemcpyHostToDevice, st));
    }
    PW_CUDA(cudaStreamSynchronize(st));
    return PW_OK;
}

extern "C" pw_status pw_batch_create(pw_mesh *const *meshes, int n, void *stream, pw_batch **out) {
    if (!out) return pw_fail(PW_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!meshes || n < 1) return pw_fail(PW_ERR_ARG, "need at least one mesh");
    for (int q = 0; q < n; q++) {
        if (!meshes[q]) return pw_fail(PW_ERR_ARG, "mesh %d is NULL", q);
        if (meshes[q]->dtype != PW_F32) return pw_fail(PW_ERR_DTYPE, "batched advection needs PW_F32 meshes");
        if (meshes[q]->device != meshes[0]->device) return pw_fail(PW_ERR_ARG, "meshes on different devices");
    }
    pw_batch *bb = new (std::nothrow) pw_batch();
    if (!bb) return pw_fail(PW_ERR_NOMEM, "host allocation");
    pw_batch_impl &b = bb->impl;
    b.n = n;
    b.meshes.assign(meshes, meshes + n);
    for (int f = 0; f < 6; f++) b.ptr[f].assign(n, nullptr);
    cudaError_t e;
    if ((e = cudaMalloc(&b.dev, sizeof(PwBatchMember) * n)) != cudaSuccess ||
        (e = cudaMalloc(&b.counter, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&b.status, sizeof(int) + 3 * sizeof(void *) * n + 64)) != cudaSuccess) {
        pw_batch_destroy(bb);
        return pw_cuda_fail(e, "cudaMalloc (batch)");
    }
    cudaStream_t st = (cudaStream_t)stream;
    if ((e = cudaMemsetAsync(b.status, 0, sizeof(int), st)) != cudaSuccess) {
        pw_batch_destroy(bb);
        return pw_cuda_fail(e, "batch status");
    }
    pw_status s = pw_batch_build(b, st);
    if (s != PW_OK) {
        pw_batch_destroy(bb);
        return s;
    }
    *out = bb;
    return PW_OK;
}

extern "C" void pw_batch_destroy(pw_batch *bb) {
    if (!bb) return;
    cudaFree(bb->impl.dev);
    cudaFree(bb->impl.counter);
    cudaFree(bb->impl.status);
    delete bb;
}

extern "C" pw_status pw_batch_set_fields(pw_batch *bb, void *const *u, void *const *v, void *const *w,
                                         void *const *su, void *const *sv, void *const *sw, void *stream) {
    if (!bb) return pw_fail(PW_ERR_ARG, "batch is NULL");
    pw_batch_impl &b = bb->impl;
    void *const *lists[6] = {u, v, w, su, sv, sw};
    const char *nm[6] = {"u", "v", "w", "su", "sv", "sw"};
    for (int f = 0; f < 6; f++) {
        if (!lists[f]) return pw_fail(PW_ERR_ARG, "%s list is NULL", nm[f]);
        for (int q = 0; q < b.n; q++) {
            char name[32];
            snprintf(name, sizeof(name), "%s[%d]", nm[f], q);
            pw_status s = pw_check_ptr(lists[f][q], name);
            if (s != PW_OK) return s;
        }
    }
    for (int f = 0; f < 6; f++) b.ptr[f].assign(lists[f], lists[f] + b.n);
    b.bound = true;
    pw_status s = pw_batch_build(b, (cudaStream_t)stream);
    if (s != PW_OK) b.bound = false;
    return s;
}

extern "C" pw_status pw_batch_set_tile(pw_batch *bb, int threads, int tile_i, void *stream) {
    if (!bb) return pw_fail(PW_ERR_ARG, "batch is NULL");
    if (threads < 32 || threads > 512 || threads % 32 != 0 || tile_i < 1 || tile_i > 1 << 20)
        return pw_fail(PW_ERR_ARG, "threads must be a multiple of 32 in 32..512 and tile_i >= 1");
    pw_batch_impl &b = bb->impl;
    const int ot = b.threads, oi = b.tile_i;
    b.threads = threads;
    b.tile_i = tile_i;
    pw_status s = pw_batch_build(b, (cudaStream_t)stream);
    if (s != PW_OK) {
        b.threads = ot;
        b.tile_i = oi;
        pw_batch_build(b, (cudaStream_t)stream);
    }
    return s;
}

extern "C" pw_status pw_batch_set_schedule(pw_batch *bb, int persistent, void *stream) {
    if (!bb) return pw_fail(PW_ERR_ARG, "batch is NULL");
    if (persistent != 0 && persistent != 1) return pw_fail(PW_ERR_ARG, "persistent must be 0 or 1");
    pw_batch_impl &b = bb->impl;
    const int old = b.persistent;
    b.persistent = persistent;
    pw_status s = pw_batch_build(b, (cudaStream_t)stream);
    if (s != PW_OK) {
        b.persistent = old;
        pw_batch_build(b, (cudaStream_t)stream);
    }
    return s;
}

static pw_status pw_batch_launch(pw_batch_impl &b, int beta, cudaStream_t st) {
    PW_CUDA(cudaMemsetAsync(b.counter, 0, sizeof(int), st));
    pw_batch_kernel<<<b.grid, b.threads, b.smem, st>>>(b.dev, b.n, b.total_tiles, b.counter, b.status, beta,
                                                       b.persistent);
    PW_CUDA(cudaGetLastError());
    return PW_OK;
}

extern "C" pw_status pw_advect_batched(pw_batch *bb, int beta, void *stream) {
    if (!bb) return pw_fail(PW_ERR_ARG, "batch is NULL");
    if (beta != 0 && beta != 1) return pw_fail(PW_ERR_ARG, "beta must be 0 or 1");
    if (!bb->impl.bound) return pw_fail(PW_ERR_ARG, "no fields bound (pw_batch_set_fields)");
    return pw_batch_launch(bb->impl, beta, (cudaStream_t)stream);
}

extern "C" pw_status pw_batch_halo(pw_batch *bb, void *stream) {
    if (!bb) return pw_fail(PW_ERR_ARG, "batch is NULL");
    pw_batch_impl &b = bb->impl;
    if (!b.bound) return pw_fail(PW_ERR_ARG, "no fields bound (pw_batch_set_fields)");
    const int warps = 8;
    pw_batch_halo_kernel<<<(b.halo_cols + warps - 1) / warps, warps * 32, 0, (cudaStream_t)stream>>>(
        b.dev, b.n, b.halo_cols, pw_batch_field_table(b));
    PW_CUDA(cudaGetLastError());
    return PW_OK;
}

extern "C" pw_status pw_batch_status(pw_batch *bb, int clear, void *stream, int *status) {
    if (!bb || !status) return pw_fail(PW_ERR_ARG, "batch and status must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    PW_CUDA(cudaMemcpyAsync(&h, bb->impl.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (clear) PW_CUDA(cudaMemsetAsync(bb->impl.status, 0, sizeof(int), st));
    PW_CUDA(cudaStreamSynchronize(st));
    *status = h;
    return PW_OK;
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
static bool pw_cache_lookup(const char *path, const std::string &key, int *a, int *b) {
    if (!path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        char k[400];
        int x, y;
        float ms;
        if (sscanf(line, "%399[^\t]\t%d\t%d\t%f", k, &x, &y, &ms) == 4 && key == k) {
            *a = x;
            *b = y;
            found = true;
        }
    }
    fclose(f);
    return found;
}

static pw_status pw_cache_store(const char *path, const std::string &key, int a, int b, float ms) {
    if (!path) return PW_OK;
    std::vector<std::string> keep;
    if (FILE *f = fopen(path, "r")) {
        char line[512];
        while (fgets(line, sizeof(line), f)) {
            if (strncmp(line, key.c_str(), key.size()) == 0 && line[key.size()] == '\t') continue;
            keep.push_back(line);
        }
        fclose(f);
    }
    FILE *f = fopen(path, "w");
    if (!f) return pw_fail(PW_ERR_IO, "cannot write autotune cache %s", path);
    for (auto &l : keep) fputs(l.c_str(), f);
    fprintf(f, "%s\t%d\t%d\t%.5f\n", key.c_str(), a, b, ms);
    fclose(f);
    return PW_OK;
}

template <typename F>
static pw_status pw_time(F launch, cudaStream_t st, float *ms_out) {
    cudaEvent_t e0, e1;
    PW_CUDA(cudaEventCreate(&e0));
    PW_CUDA(cudaEventCreate(&e1));
    pw_status s = launch();
    if (s == PW_OK) {
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && s == PW_OK; r++) s = launch();
        cudaEventRecord(e1, st);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) s = pw_cuda_fail(e, "autotune timing");
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        *ms_out = ms / 3;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return s;
}

extern "C" pw_status pw_autotune(pw_mesh *m, const void *u, const void *v, const void *w, void *su,
                                 void *sv, void *sw, const char *cache_path, void *stream, float *best_ms) {
    if (!m) return pw_fail(PW_ERR_ARG, "mesh is NULL");
    const void *p[6] = {u, v, w, su, sv, sw};
    const char *nm[6] = {"u", "v", "w", "su", "sv", "sw"};
    for (int q = 0; q < 6; q++) {
        pw_status s = pw_check_ptr(p[q], nm[q]);
        if (s != PW_OK) return s;
    }
    cudaStream_t st = (cudaStream_t)stream;
    char key[256];
    snprintf(key, sizeof(key), "mesh %d %d %d dtype=%d algo=%d sms=%d", m->nx, m->ny, m->nz, (int)m->dtype,
             (int)m->algo, m->num_sms);
    int tj = 0, ti = 0;
    if (pw_cache_lookup(cache_path, key, &tj, &ti)) {
        pw_status s = pw_mesh_set_tile(m, tj, ti);
        if (best_ms) *best_ms = -1.0f;
        return s;
    }
    std::vector<int> cj, ci = {16, 32, 64, 128, 256};
    if (m->dtype == PW_F64 && m->algo == PW_ALGO_F64_SPLIT) cj = {4, 8};
    else if (m->dtype == PW_F64) cj = {2, 4, 8};
    else cj = {2, 4, 8};
    float best = 1e30f;
    int bj = m->tile_j, bi = m->tile_i;
    const int was_auto = m->tile_i_auto;
    m->tile_i_auto = 0;  // time the candidates as given
    for (int a : cj)
        for (int c : ci) {
            float ms = 0;
            pw_status s = pw_time([&] { return pw_launch_advect(m, u, v, w, su, sv, sw, 0, st, a, c); }, st, &ms);
            if (s == PW_ERR_SHAPE) continue;  // candidate does not fit this mesh
            if (s != PW_OK) {
                m->tile_i_auto = was_auto;
                return s;
            }
            if (ms < best) {
                best = ms;
                bj = a;
                bi = c;
            }
        }
    if (best >= 1e30f) {
        m->tile_i_auto = was_auto;
        return pw_fail(PW_ERR_SHAPE, "no tile candidate fits this mesh");
    }
    m->tile_j = bj;
    m->tile_i = bi;
    if (best_ms) *best_ms = best;
    return pw_cache_store(cache_path, key, bj, bi, best);
}

extern "C" pw_status pw_batch_autotune(pw_batch *bb, const char *cache_path, void *stream, float *best_ms) {
    if (!bb) return pw_fail(PW_ERR_ARG, "batch is NULL");
    pw_batch_impl &b = bb->impl;
    if (!b.bound) return pw_fail(PW_ERR_ARG, "no fields bound (pw_batch_set_fields)");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long hsh = 1469598103934665603ull;
    for (auto *m : b.meshes) {
        const int d[3] = {m->nx, m->ny, m->nz};
        for (int x : d) hsh = (hsh ^ (unsigned)x) * 1099511628211ull;
    }
    char key[256];
    snprintf(key, sizeof(key), "batch n=%d shapes=%016llx sms=%d", b.n, hsh, b.meshes[0]->num_sms);
    // cached: threads, tile_i, and the schedule encoded in the sign of tile_i
    // (negative: one CTA per tile)
    int th = 0, ti = 0;
    if (pw_cache_lookup(cache_path, key, &th, &ti)) {
        b.threads = th;
        b.tile_i = ti < 0 ? -ti : ti;
        b.persistent = ti < 0 ? 0 : 1;
        if (best_ms) *best_ms = -1.0f;
        return pw_batch_build(b, st);
    }
    // every CTA size that is a whole number of warps (it sets how many rows of
    // each member's columns a tile holds, so how many lanes idle), three march
    // lengths, both schedules
    float best = 1e30f;
    int bt = b.threads, bi = b.tile_i, bp = b.persistent;
    for (int p : {1, 0})
        for (int t = 64; t <= 512; t += 32)
            for (int c : {32, 64, 128}) {
                b.threads = t;
                b.tile_i = c;
                b.persistent = p;
                pw_status s = pw_batch_build(b, st);
                if (s == PW_ERR_SHAPE) continue;
                if (s != PW_OK) return s;
                float ms = 0;
                s = pw_time([&] { return pw_batch_launch(b, 0, st); }, st, &ms);
                if (s != PW_OK) return s;
                if (ms < best) {
                    best = ms;
                    bt = t;
                    bi = c;
                    bp = p;
                }
            }
    b.threads = bt;
    b.tile_i = bi;
    b.persistent = bp;
    pw_status s = pw_batch_build(b, st);
    if (s != PW_OK) return s;
    if (best_ms) *best_ms = best;
    bi = bp ? bi : -bi;
    return pw_cache_store(cache_path, key, bt, bi, best);
}
