// pw_scalars.cu -- PW advection of cell-centred scalars (theta and the q fields)
// by the wind (u, v, w), many scalars per launch.
//
// The advection component serves every advected field with the same wind:
// u, v and w are shared between the kernels, the scalars are the further
// fields to advect (paper section 3).  A scalar phi sits at the cell centre,
// so the wind components on its six faces are used as they are:
//   s = hx [u(i-1) phi(i-1) - u(i) phi(i+1)] + hy [v(j-1) phi(j-1) - v(j) phi(j+1)]
//     + hz1(k) w(k-1) phi(k-1) - hz2(k) w(k) phi(k+1)
// with hx = 0.5/dx = 2 tcx, hy = 2 tcy, hz1 = 2 tzc1, hz2 = 2 tzc2 (doubling is
// exact in floating point), w(-1) = 0 at the ground and w(nz-1) = 0 at the lid.
//
// Layout of the work: the x-march of pw_march.cuh.  A CTA owns tile_j rows, one
// k chunk and a group of G scalars; a ring of NS shared-memory slots holds the
// (j,k) planes of u, v, w and the G scalars, fetched by TMA (zero fill beyond
// nz and at the lid, whose level the w tensor map leaves out).  The wind is
// read once per group, so a launch moves (3 + 2 G) values per point and group
// instead of 5 per point and scalar.
#include <algorithm>
#include <type_traits>

#include "pw_march.cuh"

#define PW_SCALAR_NS 3    // planes i, i+1 and the one in flight
#define PW_SCALAR_GMAX 6  // scalars per CTA at most

struct PwScalarSet {
    CUtensorMap phi[PW_MAX_SCALARS];  // one per scalar, box {kb, tj+2, 1}
    void *out[PW_MAX_SCALARS];        // sources, same layout as the fields
};

struct PwScalarGeom {
    PwGeom g;     // march geometry (field_stride: elements between fields of a slot)
    int nkc;      // k chunks
    int group;    // scalars per CTA
    int n;        // scalars in the launch
};

template <typename TS, typename TC, int KV>
__device__ __forceinline__ void pw_slab(const TS *row, int kk, TC (&x)[KV]) {
    SlabLoad<TS, TC, KV>::run(row + kk, x);
}

// GMAX: most scalars a CTA carries (their x window lives in registers).
// STEP: write phi + dt s (the forward Euler step fused into the stencil; phi is
// the centre value already in registers) in the field type, at the column and
// at its periodic halo images, instead of the source s.
template <typename TS, typename TC, typename TO, int KV, int NS, int GMAX, bool STEP = false>
__global__ void __launch_bounds__(512)
pw_scalar_march(const __grid_constant__ CUtensorMap mu, const __grid_constant__ CUtensorMap mv,
                const __grid_constant__ CUtensorMap mw, const __grid_constant__ PwScalarSet set,
                const TC *__restrict__ coef, const PwScalarGeom sg, int beta, int *__restrict__ status,
                double dt = 0.0) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if (pw_cta_failed(status)) return;
    const PwGeom &g = sg.g;
    const int kchunk = blockIdx.z % sg.nkc, grp = blockIdx.z / sg.nkc;
    const int s0 = grp * sg.group;
    const int G = min(sg.group, sg.n - s0);  // scalars of this CTA (<= GMAX)
    const int NF = 3 + G;                    // fields in a slot
    const int j0 = blockIdx.x * g.tj, i0 = blockIdx.y * g.ti, k0 = kchunk * g.kc;
    const int fs = g.field_stride;
    const size_t slot_elems = (size_t)(3 + sg.group) * fs;
    TS *planes = reinterpret_cast<TS *>(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + NS * slot_elems * sizeof(TS));

    const int nkt = g.kc / KV;
    const int tid = threadIdx.x, lane = tid & 31;
    const int tk = tid % nkt, tj = tid / nkt;
    const int i_end = min(i0 + g.ti, g.nx);
    const int nplanes = i_end - i0 + 2;
    const uint32_t plane_bytes = (uint32_t)NF * (uint32_t)g.plane_elems * (uint32_t)sizeof(TS);
    const int kbase = k0 + tk * KV, kk = g.h + tk * KV;
    const int j = j0 + tj;
    const bool in_tile = tj < g.tj;
    const int tjc = in_tile ? tj : g.tj - 1;
    const bool active = in_tile && (j < g.ny) && (kbase < g.nz);
    const int nvalid = g.nz - kbase;
    const int wbase = tid & ~31;
    const unsigned mask = (int)blockDim.x - wbase >= 32 ? 0xffffffffu
                                                         : ((1u << ((int)blockDim.x - wbase)) - 1u);
    const bool lo_shfl = tk > 0 && lane > 0;
    const bool hi_shfl = tk < nkt - 1 && lane < 31 && tid + 1 < (int)blockDim.x;

    if (tid == 0) {
        pw_prefetch_map(&mu);
        pw_prefetch_map(&mv);
        pw_prefetch_map(&mw);
        for (int q = 0; q < G; q++) pw_prefetch_map(&set.phi[s0 + q]);
        for (int s = 0; s < NS; s++) pw_mbar_init(&bars[s], 1);
        pw_fence_barrier_init();
    }
    __syncthreads();

    auto slot = [&](int p) { return planes + (size_t)(p % NS) * slot_elems; };
    auto issue = [&](int p) {
        const int s = p % NS;
        TS *dst = slot(p);
        pw_mbar_expect_tx(&bars[s], plane_bytes);
        const int c0 = k0 - g.h, c1 = j0 + 1, c2 = i0 + 1 + p;  // (k, j-1, i-1+p) + halo offset
        pw_tma_load_3d(dst, &mu, c0, c1, c2, &bars[s]);
        pw_tma_load_3d(dst + fs, &mv, c0, c1, c2, &bars[s]);
        pw_tma_load_3d(dst + 2 * fs, &mw, c0, c1, c2, &bars[s]);
        for (int q = 0; q < G; q++)
            pw_tma_load_3d(dst + (size_t)(3 + q) * fs, &set.phi[s0 + q], c0, c1, c2, &bars[s]);
    };
    int issued = 0;
    if (tid == 0) {
        for (int p = 0; p < min(NS, nplanes); p++) issue(p);
        issued = min(NS, nplanes);
    }
    auto give_up = [&](int waited) {
        if (tid == 0) {
            for (int p = waited; p < issued; p++)
                if (!pw_mbar_wait_bounded(&bars[p % NS], (uint32_t)((p / NS) & 1), PW_DRAIN_CYCLES)) break;
            atomicExch(status, (int)PW_ERR_TIMEOUT);
        }
    };

    // vertical coefficients of this thread's levels, doubled (exact): hz1, hz2
    TC c1[KV], c2[KV];
#pragma unroll
    for (int m = 0; m < KV; m++) {
        const int k = kbase + m;
        const bool in = k < g.nz;
        c1[m] = in ? TC(2) * coef[k] : TC(0);
        c2[m] = in ? TC(2) * coef[g.nz + k] : TC(0);
    }
    const TC hx = TC(2) * pw_geom_c<TC>(g.tcx, g.ftcx), hy = TC(2) * pw_geom_c<TC>(g.tcy, g.ftcy);
    const TC tdt = (TC)dt;
    const int L = g.kb;
    const int rS = tjc * L, rC = (tjc + 1) * L, rN = (tjc + 2) * L;

    // the x window: u and every scalar at column i-1 (centre row), in registers,
    // so the ring holds only planes i, i+1 and the one in flight
    TC uM[KV], pM[GMAX][KV];
    {
        const bool ok = pw_mbar_wait_bounded(&bars[0], 0);
        if (!__syncthreads_and(ok)) {
            give_up(0);
            return;
        }
        const TS *P0 = slot(0);
        pw_slab<TS, TC, KV>(P0 + rC, kk, uM);
#pragma unroll
        for (int s = 0; s < GMAX; s++)
            if (s < G) pw_slab<TS, TC, KV>(P0 + (size_t)(3 + s) * fs + rC, kk, pM[s]);
    }
    int waited = 1;  // planes 0 .. waited-1 have landed
    for (int i = i0; i < i_end; i++) {
        const int q = i - i0 + 1;  // plane of column i
        bool ok = true;
        while (ok && waited <= q + 1) {
            ok = pw_mbar_wait_bounded(&bars[waited % NS], (uint32_t)((waited / NS) & 1));
            if (ok) waited++;
        }
        if (!__syncthreads_and(ok)) {
            give_up(waited);
            return;
        }
        // every thread is past step i-1 (planes q-1 and q) and the window load:
        // the slot of plane q-1 is free
        if (tid == 0 && q - 1 + NS < nplanes) {
            issue(q - 1 + NS);
            issued = q + NS;
        }
        const TS *Pc = slot(q), *Pp = slot(q + 1);
        TC uC[KV], vS[KV], vC[KV], wC[KV + 2];
        pw_slab<TS, TC, KV>(Pc + rC, kk, uC);
        pw_slab<TS, TC, KV>(Pc + fs + rS, kk, vS);
        pw_slab<TS, TC, KV>(Pc + fs + rC, kk, vC);
        pw_col_edges<TS, TC, KV>(Pc + 2 * fs + rC, kk, wC, mask, lo_shfl, hi_shfl, true, false);
        const long long off = (long long)(i + 2) * g.si + (long long)(j + 2) * g.sj + kbase;
#pragma unroll
        for (int s = 0; s < GMAX; s++) {
            if (s < G) {
                const size_t fo = (size_t)(3 + s) * fs;
                TC pP[KV], pS[KV], pN[KV], pC[KV + 2];
                pw_slab<TS, TC, KV>(Pp + fo + rC, kk, pP);
                pw_slab<TS, TC, KV>(Pc + fo + rS, kk, pS);
                pw_slab<TS, TC, KV>(Pc + fo + rN, kk, pN);
                pw_col_edges<TS, TC, KV>(Pc + fo + rC, kk, pC, mask, lo_shfl, hi_shfl, true, true);
                if (active) {
                    TO r[KV];
#pragma unroll
                    for (int m = 0; m < KV; m++) {
                        TC x = hx * (uM[m] * pM[s][m] - uC[m] * pP[m]);
                        x = x + hy * (vS[m] * pS[m] - vC[m] * pN[m]);
                        x = x + c1[m] * wC[m] * pC[m];
                        x = x - c2[m] * wC[m + 1] * pC[m + 2];
                        r[m] = STEP ? (TO)(pC[m + 1] + tdt * x) : (TO)x;
                    }
                    if (STEP)
                        pw_store_images<TO, KV>(reinterpret_cast<TO *>(set.out[s0 + s]), i, j, kbase, r, nvalid,
                                                g.nx, g.ny, g.si, g.sj);
                    else
                        pw_store<TO, KV>(reinterpret_cast<TO *>(set.out[s0 + s]) + off, r, nvalid, beta);
                }
#pragma unroll
                for (int m = 0; m < KV; m++) pM[s][m] = pC[m + 1];
            }
        }
#pragma unroll
        for (int m = 0; m < KV; m++) uM[m] = uC[m];
    }
    __syncthreads();
    if (tid == 0)
        for (int s = 0; s < NS; s++) pw_mbar_inval(&bars[s]);
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
template <typename TS, typename TC, typename TO, int KV, bool STEP = false>
static pw_status pw_launch_scalars(const pw_mesh *m, const void *u, const void *v, const void *w, int n,
                                   const void *const *phi, void *const *sphi, int beta, cudaStream_t st,
                                   int tile_j, int tile_i, int group, double dt = 0.0) {
    constexpr int NS = PW_SCALAR_NS;
    PwScalarGeom sg;
    PwGeom &g = sg.g;
    g.nx = m->nx;
    g.ny = m->ny;
    g.nz = m->nz;
    g.nzp = m->nzp;
    g.h = 16 / (int)sizeof(TS);
    const int unit = std::max(KV, g.h);  // KV and h are powers of two
    const int kc_one = (m->nz + unit - 1) / unit * unit;
    const int kc_max = sizeof(TS) == 8 ? 64 : 128;  // keeps a slot of a few scalars small
    g.kc = kc_one <= kc_max ? kc_one : kc_max;
    g.kb = g.kc + 2 * g.h;
    // rows per CTA: as asked, but no more than 512 threads (long columns)
    tile_j = tile_j < 512 / (g.kc / KV) ? tile_j : 512 / (g.kc / KV);
    if (tile_j < 1) tile_j = 1;
    g.tj = tile_j;
    g.ns = NS;
    g.plane_elems = (tile_j + 2) * g.kb;
    const int per128 = 128 / (int)sizeof(TS);
    g.field_stride = (g.plane_elems + per128 - 1) / per128 * per128;
    g.si = m->si;
    g.sj = m->sj;
    g.tcx = m->tcx;
    g.tcy = m->tcy;
    g.ftcx = (float)m->tcx;
    g.ftcy = (float)m->tcy;
    const int threads = (g.kc / KV) * tile_j;
    if (threads > 512)
        return pw_fail(PW_ERR_SHAPE, "scalars: tile_j=%d needs %d threads (> 512)", tile_j, threads);
    const size_t field_bytes = (size_t)NS * g.field_stride * sizeof(TS);
    // scalars per CTA: as many as fit beside the wind in one CTA's shared
    // memory (at most PW_SCALAR_GMAX, whose x window is held in registers),
    // then balanced over the groups; fewer groups means fewer reads of the wind
    if (group <= 0) {
        const long fit = (long)(226 * 1024) / (long)field_bytes - 3;
        group = (int)std::max(1L, std::min((long)std::min(n, PW_SCALAR_GMAX), fit));
        const int ngroups = (n + group - 1) / group;
        group = (n + ngroups - 1) / ngroups;
    }
    group = std::min(std::min(group, n), PW_SCALAR_GMAX);
    sg.group = group;
    sg.n = n;
    sg.nkc = (m->nz + g.kc - 1) / g.kc;
    const size_t smem = field_bytes * (size_t)(3 + group) + (size_t)NS * sizeof(uint64_t);
    if (smem > 226 * 1024)
        return pw_fail(PW_ERR_SHAPE, "scalars: %d per CTA need %zu bytes of shared memory", group, smem);
    CUtensorMap maps[3];
    const void *f[3] = {u, v, w};
    for (int q = 0; q < 3; q++) {
        pw_status s = pw_make_field_map(&maps[q], f[q], m->dtype, m->nx, m->ny, m->nzp, pw_kdim(m->nz, q),
                                        g.kb, tile_j + 2);
        if (s != PW_OK) return s;
    }
    PwScalarSet set;
    memset(&set, 0, sizeof(set));
    for (int q = 0; q < n; q++) {
        pw_status s = pw_make_field_map(&set.phi[q], phi[q], m->dtype, m->nx, m->ny, m->nzp, m->nz, g.kb,
                                        tile_j + 2);
        if (s != PW_OK) return s;
        set.out[q] = sphi[q];
    }
    auto kern = pw_scalar_march<TS, TC, TO, KV, NS, PW_SCALAR_GMAX, STEP>;
    PW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long ngroups = (n + group - 1) / group;
    // the fill rule (the wave rule measured no faster on these many-wave grids)
    tile_i = pw_fit_tile_i(m, tile_i, (long)((m->ny + tile_j - 1) / tile_j) * sg.nkc);
    g.ti = tile_i;
    dim3 grid((unsigned)((m->ny + tile_j - 1) / tile_j), (unsigned)((m->nx + tile_i - 1) / tile_i),
              (unsigned)(sg.nkc * ngroups));
    if (grid.y > 65535 || grid.z > 65535) return pw_fail(PW_ERR_SHAPE, "grid too large; raise tile_i");
    const TC *coef = std::is_same<TC, double>::value ? reinterpret_cast<const TC *>(m->coef64 + 6 * m->nz)
                                                     : reinterpret_cast<const TC *>(m->coef32);
    kern<<<grid, threads, smem, st>>>(maps[0], maps[1], maps[2], set, coef, sg, beta, m->status, dt);
    PW_CUDA(cudaGetLastError());
    return PW_OK;
}

pw_status pw_launch_scalars_split(const pw_mesh *m, const void *u, const void *v, const void *w, int n,
                                  const void *const *phi, void *const *sphi, int beta, cudaStream_t st,
                                  int tile_j, int tile_i, int group, bool step = false, double dt = 0.0);

pw_status pw_launch_advect_scalars(const pw_mesh *m, const void *u, const void *v, const void *w, int n,
                                   const void *const *phi, void *const *sphi, int beta, cudaStream_t st,
                                   int tile_j, int tile_i, int group) {
    switch (m->dtype) {
        case PW_F64:
            if (m->algo == PW_ALGO_F64_SPLIT)
                return pw_launch_scalars_split(m, u, v, w, n, phi, sphi, beta, st, tile_j, tile_i, group);
            return pw_launch_scalars<double, double, double, 2>(m, u, v, w, n, phi, sphi, beta, st, tile_j,
                                                                tile_i, group);
        case PW_F32:
            return pw_launch_scalars<float, float, float, 4>(m, u, v, w, n, phi, sphi, beta, st, tile_j,
                                                             tile_i, group);
        case PW_BF16:
            return pw_launch_scalars<__nv_bfloat16, float, float, 4>(m, u, v, w, n, phi, sphi, beta, st,
                                                                     tile_j, tile_i, group);
        case PW_BF16_OUT:
            return pw_launch_scalars<__nv_bfloat16, float, __nv_bfloat16, 4>(m, u, v, w, n, phi, sphi, beta, st,
                                                                             tile_j, tile_i, group);
    }
    return pw_fail(PW_ERR_DTYPE, "unknown dtype");
}

// checks shared by the scalar entry points: pointers, count, no aliasing
static pw_status pw_check_scalar_args(const void *u, const void *v, const void *w, int n,
                                      const void *const *phi, void *const *out) {
    if (n < 1 || n > PW_MAX_SCALARS) return pw_fail(PW_ERR_ARG, "n = %d scalars (1..%d)", n, PW_MAX_SCALARS);
    if (!phi || !out) return pw_fail(PW_ERR_ARG, "scalar pointer arrays are NULL");
    const void *wind[3] = {u, v, w};
    const char *wn[3] = {"u", "v", "w"};
    for (int q = 0; q < 3; q++) {
        pw_status s = pw_check_ptr(wind[q], wn[q]);
        if (s != PW_OK) return s;
    }
    for (int a = 0; a < n; a++) {
        pw_status s = pw_check_ptr(phi[a], "phi[a]");
        if (s != PW_OK) return s;
        s = pw_check_ptr(out[a], "out[a]");
        if (s != PW_OK) return s;
        for (int q = 0; q < 3; q++)
            if (out[a] == wind[q]) return pw_fail(PW_ERR_ARG, "output %d aliases %s", a, wn[q]);
        for (int b = 0; b < n; b++) {
            if (out[a] == phi[b]) return pw_fail(PW_ERR_ARG, "output %d aliases phi[%d]", a, b);
            if (b > a && out[a] == out[b]) return pw_fail(PW_ERR_ARG, "outputs %d and %d alias", a, b);
        }
    }
    return PW_OK;
}

extern "C" pw_status pw_advect_scalars(const pw_mesh *m, const void *u, const void *v, const void *w, int n,
                                       const void *const *phi, void *const *sphi, int beta, void *stream) {
    if (!m) return pw_fail(PW_ERR_ARG, "mesh is NULL");
    if (beta != 0 && beta != 1) return pw_fail(PW_ERR_ARG, "beta must be 0 or 1");
    pw_status s = pw_check_scalar_args(u, v, w, n, phi, sphi);
    if (s != PW_OK) return s;
    return pw_launch_advect_scalars(m, u, v, w, n, phi, sphi, beta, (cudaStream_t)stream, m->tile_j,
                                    m->tile_i, 0);
}

pw_status pw_launch_scalars_step(const pw_mesh *m, const void *u, const void *v, const void *w, int n,
                                 const void *const *phi, void *const *phin, double dt, cudaStream_t st,
                                 int tile_j, int tile_i) {
    switch (m->dtype) {
        case PW_F64:
            if (m->algo == PW_ALGO_F64_SPLIT)
                return pw_launch_scalars_split(m, u, v, w, n, phi, phin, 0, st, tile_j, tile_i, 0, true, dt);
            return pw_launch_scalars<double, double, double, 2, true>(m, u, v, w, n, phi, phin, 0, st, tile_j,
                                                                      tile_i, 0, dt);
        case PW_F32:
            return pw_launch_scalars<float, float, float, 4, true>(m, u, v, w, n, phi, phin, 0, st, tile_j,
                                                                   tile_i, 0, dt);
        case PW_BF16:
        case PW_BF16_OUT:  // the new state has the field type either way
            return pw_launch_scalars<__nv_bfloat16, float, __nv_bfloat16, 4, true>(m, u, v, w, n, phi, phin, 0,
                                                                                   st, tile_j, tile_i, 0, dt);
    }
    return pw_fail(PW_ERR_DTYPE, "unknown dtype");
}

extern "C" pw_status pw_advect_scalars_step(const pw_mesh *m, const void *u, const void *v, const void *w,
                                            int n, const void *const *phi, void *const *phin, double dt,
                                            void *stream) {
    if (!m) return pw_fail(PW_ERR_ARG, "mesh is NULL");
    if (!(dt == dt) || dt - dt != 0.0) return pw_fail(PW_ERR_ARG, "dt must be finite");
    pw_status s = pw_check_scalar_args(u, v, w, n, phi, phin);
    if (s != PW_OK) return s;
    return pw_launch_scalars_step(m, u, v, w, n, phi, phin, dt, (cudaStream_t)stream, m->tile_j, m->tile_i);
}
