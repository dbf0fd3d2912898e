// pw_advect.cu -- forward PW stencil launches: FP64 (native), FP32 and
// BF16-in/FP32-out through the x-march of pw_march.cuh; FP64 split path in
// pw_advect_split.cu.
#include <algorithm>
#include <type_traits>

#include "pw_march.cuh"


template <typename TS, typename TC, typename TO, int KV>
__global__ void __launch_bounds__(512)
pw_advect_march(const __grid_constant__ CUtensorMap mu, const __grid_constant__ CUtensorMap mv,
                const __grid_constant__ CUtensorMap mw, TO *__restrict__ su, TO *__restrict__ sv,
                TO *__restrict__ sw, const TC *__restrict__ coef, const PwGeom g, int beta,
                int *__restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if (pw_cta_failed(status)) return;  // sticky failure: do nothing until cleared
    pw_march_tile<TS, TC, TO, KV, PW_MARCH_NS>(&mu, &mv, &mw, su, sv, sw, coef, g, beta, status,
                                               smem_raw, blockIdx.x * g.tj, blockIdx.y * g.ti,
                                               blockIdx.z * g.kc);
}

// the forward Euler step fused into the stencil: xn = x + dt S(x), halos included
template <typename TS, typename TC, int KV>
__global__ void __launch_bounds__(512)
pw_step_march(const __grid_constant__ CUtensorMap mu, const __grid_constant__ CUtensorMap mv,
              const __grid_constant__ CUtensorMap mw, TS *__restrict__ un, TS *__restrict__ vn,
              TS *__restrict__ wn, const TC *__restrict__ coef, const PwGeom g, double dt,
              int *__restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if (pw_cta_failed(status)) return;
    pw_march_tile<TS, TC, TS, KV, PW_MARCH_NS, true>(&mu, &mv, &mw, un, vn, wn, coef, g, 0, status, smem_raw,
                                                     blockIdx.x * g.tj, blockIdx.y * g.ti, blockIdx.z * g.kc, dt);
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
static int pw_lcm(int a, int b) {
    int x = a, y = b;
    while (y) {
        int t = x % y;
        x = y;
        y = t;
    }
    return a / x * b;
}

template <typename TS, typename TC, typename TO, int KV, bool STEP = false>
static pw_status pw_launch_march(const pw_mesh *m, const void *u, const void *v, const void *w,
                                 void *su, void *sv, void *sw, int beta, cudaStream_t st,
                                 int tile_j, int tile_i, int ns, double dt = 0.0) {
    PwGeom g;
    g.nx = m->nx;
    g.ny = m->ny;
    g.nz = m->nz;
    g.nzp = m->nzp;
    g.h = 16 / (int)sizeof(TS);
    int unit = pw_lcm(KV, g.h);
    int kc_one = (m->nz + unit - 1) / unit * unit;
    g.kc = (kc_one + 2 * g.h <= 256) ? kc_one : 128;
    g.kb = g.kc + 2 * g.h;
    // rows per CTA: as asked, but no more than 512 threads (long columns)
    tile_j = std::max(1, std::min(tile_j, 512 / (g.kc / KV)));
    g.tj = tile_j;
    const long tiles = (long)((m->ny + tile_j - 1) / tile_j) * ((m->nz + g.kc - 1) / g.kc);
    g.ns = ns;
    g.plane_elems = (tile_j + 2) * g.kb;
    int per128 = 128 / (int)sizeof(TS);
    g.field_stride = (g.plane_elems + per128 - 1) / per128 * per128;
    g.si = m->si;
    g.sj = m->sj;
    g.tcx = m->tcx;
    g.tcy = m->tcy;
    g.ftcx = (float)m->tcx;
    g.ftcy = (float)m->tcy;
    int threads = (g.kc / KV) * tile_j;
    if (threads > 512)
        return pw_fail(PW_ERR_SHAPE, "tile_j=%d needs %d threads (> 512) for k chunk %d", tile_j,
                       threads, g.kc);
    size_t smem = (size_t)ns * 3 * g.field_stride * sizeof(TS) + (size_t)ns * sizeof(uint64_t);
    if (smem > 226 * 1024) return pw_fail(PW_ERR_SHAPE, "tile needs %zu bytes of shared memory", smem);
    CUtensorMap maps[3];
    const void *f[3] = {u, v, w};
    for (int q = 0; q < 3; q++) {
        pw_status s = pw_make_field_map(&maps[q], f[q], m->dtype, m->nx, m->ny, m->nzp, pw_kdim(m->nz, q),
                                        g.kb, tile_j + 2);
        if (s != PW_OK) return s;
    }
    const auto kern = [] {
        if constexpr (STEP) return pw_step_march<TS, TC, KV>;
        else return pw_advect_march<TS, TC, TO, KV>;
    }();
    PW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // a CTA marches ti columns from ti + 2 planes
    tile_i = pw_pick_tile_i(m, tile_i, tiles, pw_slots(m, kern, threads, smem), 2);
    g.ti = tile_i;
    dim3 grid((unsigned)((m->ny + tile_j - 1) / tile_j), (unsigned)((m->nx + tile_i - 1) / tile_i),
              (unsigned)((m->nz + g.kc - 1) / g.kc));
    if (grid.y > 65535 || grid.z > 65535) return pw_fail(PW_ERR_SHAPE, "grid too large; raise tile_i");
    const TC *coef = std::is_same<TC, double>::value
                         ? reinterpret_cast<const TC *>(m->coef64 + 6 * m->nz)
                         : reinterpret_cast<const TC *>(m->coef32);
    if constexpr (STEP)
        kern<<<grid, threads, smem, st>>>(maps[0], maps[1], maps[2], (TS *)su, (TS *)sv, (TS *)sw, coef, g, dt,
                                          m->status);
    else
        kern<<<grid, threads, smem, st>>>(maps[0], maps[1], maps[2], (TO *)su, (TO *)sv, (TO *)sw, coef,
                                          g, beta, m->status);
    PW_CUDA(cudaGetLastError());
    return PW_OK;
}

pw_status pw_launch_advect_split(const pw_mesh *m, const void *u, const void *v, const void *w,
                                 void *su, void *sv, void *sw, int beta, cudaStream_t st,
                                 int tile_j, int tile_i);

pw_status pw_launch_advect(const pw_mesh *m, const void *u, const void *v, const void *w, void *su,
                           void *sv, void *sw, int beta, cudaStream_t st, int tile_j, int tile_i) {
    switch (m->dtype) {
        case PW_F64:
            if (m->algo == PW_ALGO_F64_SPLIT)
                return pw_launch_advect_split(m, u, v, w, su, sv, sw, beta, st, tile_j, tile_i);
            return pw_launch_march<double, double, double, 2>(m, u, v, w, su, sv, sw, beta, st,
                                                              tile_j, tile_i, PW_MARCH_NS);
        case PW_F32:
            return pw_launch_march<float, float, float, 4>(m, u, v, w, su, sv, sw, beta, st, tile_j,
                                                           tile_i, PW_MARCH_NS);
        case PW_BF16:
            return pw_launch_march<__nv_bfloat16, float, float, 4>(m, u, v, w, su, sv, sw, beta, st,
                                                                   tile_j, tile_i, PW_MARCH_NS);
        case PW_BF16_OUT:
            return pw_launch_march<__nv_bfloat16, float, __nv_bfloat16, 4>(m, u, v, w, su, sv, sw, beta, st,
                                                                           tile_j, tile_i, PW_MARCH_NS);
    }
    return pw_fail(PW_ERR_DTYPE, "unknown dtype");
}

pw_status pw_launch_step_split(const pw_mesh *m, const void *u, const void *v, const void *w, void *un,
                               void *vn, void *wn, double dt, cudaStream_t st, int tile_j, int tile_i);

pw_status pw_launch_step(const pw_mesh *m, const void *u, const void *v, const void *w, void *un, void *vn,
                         void *wn, double dt, cudaStream_t st, int tile_j, int tile_i) {
    switch (m->dtype) {
        case PW_F64:
            if (m->algo == PW_ALGO_F64_SPLIT)
                return pw_launch_step_split(m, u, v, w, un, vn, wn, dt, st, tile_j, tile_i);
            return pw_launch_march<double, double, double, 2, true>(m, u, v, w, un, vn, wn, 0, st, tile_j, tile_i,
                                                                    PW_MARCH_NS, dt);
        case PW_F32:
            return pw_launch_march<float, float, float, 4, true>(m, u, v, w, un, vn, wn, 0, st, tile_j, tile_i,
                                                                 PW_MARCH_NS, dt);
        case PW_BF16:
        case PW_BF16_OUT:  // the new state has the field type either way
            return pw_launch_march<__nv_bfloat16, float, __nv_bfloat16, 4, true>(m, u, v, w, un, vn, wn, 0, st,
                                                                                 tile_j, tile_i, PW_MARCH_NS, dt);
    }
    return pw_fail(PW_ERR_DTYPE, "unknown dtype");
}

static pw_status pw_check_fields(const void *const *p, const char *const *nm, int n) {
    for (int q = 0; q < n; q++) {
        pw_status s = pw_check_ptr(p[q], nm[q]);
        if (s != PW_OK) return s;
    }
    return PW_OK;
}

extern "C" pw_status pw_advect(const pw_mesh *m, const void *u, const void *v, const void *w,
                               void *su, void *sv, void *sw, int beta, void *stream) {
    if (!m) return pw_fail(PW_ERR_ARG, "mesh is NULL");
    if (beta != 0 && beta != 1) return pw_fail(PW_ERR_ARG, "beta must be 0 or 1");
    const void *p[6] = {u, v, w, su, sv, sw};
    const char *nm[6] = {"u", "v", "w", "su", "sv", "sw"};
    pw_status s = pw_check_fields(p, nm, 6);
    if (s != PW_OK) return s;
    for (int a = 0; a < 3; a++)
        for (int b = 3; b < 6; b++)
            if (p[a] == p[b]) return pw_fail(PW_ERR_ARG, "%s and %s alias", nm[a], nm[b]);
    if (su == sv || su == sw || sv == sw) return pw_fail(PW_ERR_ARG, "outputs alias");
    return pw_launch_advect(m, u, v, w, su, sv, sw, beta, (cudaStream_t)stream, m->tile_j, m->tile_i);
}

extern "C" pw_status pw_advect_step(const pw_mesh *m, const void *u, const void *v, const void *w, void *un,
                                    void *vn, void *wn, double dt, void *stream) {
    if (!m) return pw_fail(PW_ERR_ARG, "mesh is NULL");
    const void *p[6] = {u, v, w, un, vn, wn};
    const char *nm[6] = {"u", "v", "w", "un", "vn", "wn"};
    pw_status s = pw_check_fields(p, nm, 6);
    if (s != PW_OK) return s;
    for (int a = 0; a < 6; a++)
        for (int b = a + 1; b < 6; b++)
            if (p[a] == p[b]) return pw_fail(PW_ERR_ARG, "%s and %s alias", nm[a], nm[b]);
    if (!(dt == dt) || dt - dt != 0.0) return pw_fail(PW_ERR_ARG, "dt must be finite");
    return pw_launch_step(m, u, v, w, un, vn, wn, dt, (cudaStream_t)stream, m->tile_j, m->tile_i);
}
