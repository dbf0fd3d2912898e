// pw_adjoint.cu -- transpose of the Jacobian of the PW stencil, in gather form.
//
// Every source term is  sign * c * phi(P) * (a(Q1) + a(Q2))  attached to an
// output point m.  Its derivative sends y(m) * sign * c * (a(Q1) + a(Q2)) to
// the gradient of phi at P and y(m) * sign * c * phi(P) to the gradient of a at
// Q1 and Q2.  Instead of scattering (atomics), each thread GATHERS, for its own
// input point n, every (term, m) with P = n, Q1 = n or Q2 = n, i.e. m = n - P,
// n - Q1, n - Q2.  The incoming gradients y = (gsu, gsv, gsw) are read through
// their periodic halos, so what the forward read through a halo copy lands on
// the interior point it copies (the adjoint of the halo fill).  Ground and lid
// rules come from zeros: values at k < 0 or k >= nz, and w, gsw on the lid
// face, arrive from TMA as 0 (the tensor maps carry the logical k extent),
// which removes exactly the terms the forward drops.
//
// Same x-march as the forward kernel, with six fields (u, v, w, gsu, gsv, gsw)
// per shared-memory plane.
#include <math.h>
#include <type_traits>

#include "pw_march.cuh"  // slab loads with shuffled k edges, vector stores

// two levels per thread for FP32 (twice the threads for the same staged planes)
template <typename TC>
struct SlabLoad<float, TC, 2> {
    static __device__ __forceinline__ void run(const float *p, TC *o) {
        const float2 a = *reinterpret_cast<const float2 *>(p);
        o[0] = a.x;
        o[1] = a.y;
    }
};

struct PwAdjGeom {
    int nx, ny, nz, nzp;
    int kc, kb, h, tj, ti, ns, field_stride, plane_elems;
    long long si, sj;
    double tcx, tcy;
};


// at most 256 threads, so the six-field gather keeps its values in registers
// (shared memory limits the CTAs per SM anyway)
template <typename TS, typename TC, int KV>
__global__ void __launch_bounds__(256)
pw_adjoint_march(const __grid_constant__ CUtensorMap mu, const __grid_constant__ CUtensorMap mv,
                 const __grid_constant__ CUtensorMap mw, const __grid_constant__ CUtensorMap mgu,
                 const __grid_constant__ CUtensorMap mgv, const __grid_constant__ CUtensorMap mgw,
                 TS *__restrict__ gu, TS *__restrict__ gv, TS *__restrict__ gw,
                 const TC *__restrict__ coef, const PwAdjGeom g, TC alpha, int beta, int add_y,
                 int *__restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TS *planes = reinterpret_cast<TS *>(smem_raw);
    uint64_t *bars =
        reinterpret_cast<uint64_t *>(smem_raw + (size_t)g.ns * 6 * g.field_stride * sizeof(TS));
    const int nkt = g.kc / KV;
    const int tk = threadIdx.x % nkt, tj = threadIdx.x / nkt;
    const int j0 = blockIdx.x * g.tj, i0 = blockIdx.y * g.ti, k0 = blockIdx.z * g.kc;
    const int i_end = min(i0 + g.ti, g.nx);
    const int nplanes = i_end - i0 + 2;
    const uint32_t plane_bytes = 6u * (uint32_t)g.plane_elems * (uint32_t)sizeof(TS);
    const int kbase = k0 + tk * KV;
    const int kk = g.h + tk * KV;
    const int j = j0 + tj;
    const CUtensorMap *maps[6] = {&mu, &mv, &mw, &mgu, &mgv, &mgw};

    if (pw_cta_failed(status)) return;  // sticky failure: do nothing until cleared
    if (threadIdx.x == 0) {
        for (int f = 0; f < 6; f++) pw_prefetch_map(maps[f]);
        for (int s = 0; s < g.ns; s++) pw_mbar_init(&bars[s], 1);
        pw_fence_barrier_init();
    }
    __syncthreads();
    auto issue = [&](int p) {
        int s = p % g.ns;
        TS *dst = planes + (size_t)s * 6 * g.field_stride;
        pw_mbar_expect_tx(&bars[s], plane_bytes);
        int c0 = k0 - g.h, c1 = j0 + 1, c2 = i0 + 1 + p;
#pragma unroll
        for (int f = 0; f < 6; f++) pw_tma_load_3d(dst + f * g.field_stride, maps[f], c0, c1, c2, &bars[s]);
    };
    int issued = 0;
    if (threadIdx.x == 0) {
        for (int p = 0; p < min(g.ns, nplanes); p++) issue(p);
        issued = min(g.ns, nplanes);
    }

    // coefficients at levels kbase-1 .. kbase+KV (0 outside [0, nz))
    TC c1[KV + 2], c2[KV + 2], d1[KV + 2], d2[KV + 2];
#pragma unroll
    for (int m = 0; m < KV + 2; m++) {
        int k = kbase - 1 + m;
        bool in = k >= 0 && k < g.nz;
        c1[m] = in ? coef[k] : TC(0);
        c2[m] = in ? coef[g.nz + k] : TC(0);
        d1[m] = in ? coef[2 * g.nz + k] : TC(0);
        d2[m] = in ? coef[3 * g.nz + k] : TC(0);
    }
    const TC tcx = (TC)g.tcx, tcy = (TC)g.tcy;
    const bool active = (j < g.ny) && (kbase < g.nz);
    const int nzl = g.nz - 1;
    const int nvalid = g.nz - kbase;

    int waited = 0;
    for (int i = i0; i < i_end; i++) {
        const int q = i - i0 + 1;
        bool ok = true;
        while (waited <= q + 1 && ok) {
            ok = pw_mbar_wait_bounded(&bars[waited % g.ns], (uint32_t)((waited / g.ns) & 1));
            if (ok) waited++;
        }
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) {
                for (int p = waited; p < issued; p++)
                    if (!pw_mbar_wait_bounded(&bars[p % g.ns], (uint32_t)((p / g.ns) & 1),
                                              PW_DRAIN_CYCLES))
                        break;
                atomicExch(status, (int)PW_ERR_TIMEOUT);
            }
            return;
        }
        if (threadIdx.x == 0 && q >= 2 && q - 2 + g.ns < nplanes) {
            issue(q - 2 + g.ns);
            issued = q - 1 + g.ns;
        }

        const int fs = g.field_stride, L = g.kb;
        const TS *Pm = planes + (size_t)((q - 1) % g.ns) * 6 * fs;
        const TS *Pc = planes + (size_t)(q % g.ns) * 6 * fs;
        const TS *Pp = planes + (size_t)((q + 1) % g.ns) * 6 * fs;
        // row offsets: j-1, j, j+1
        const int rS = tj * L, rC = (tj + 1) * L, rN = (tj + 2) * L;
        enum { U = 0, V = 1, W = 2, YU = 3, YV = 4, YW = 5 };
#define COL(P, F, R, X) pw_col<TS, TC, KV, true, true>((P) + (F) * fs + (R), kk, X)
        using TOut = TS;
        TOut ru[KV], rv[KV], rw[KV];
        {   // ---------------- gu ----------------
            TC u0[KV + 2], up[KV + 2], um[KV + 2], v0[KV + 2], vp[KV + 2], vs[KV + 2], vsp[KV + 2];
            TC w0[KV + 2], wp[KV + 2], y0[KV + 2], yp[KV + 2], ym[KV + 2], yn[KV + 2], ys[KV + 2];
            TC zp[KV + 2], zps[KV + 2], z0[KV + 2], zs[KV + 2], q0[KV + 2], qp[KV + 2];
            COL(Pc, U, rC, u0); COL(Pp, U, rC, up); COL(Pm, U, rC, um);
            COL(Pc, V, rC, v0); COL(Pp, V, rC, vp); COL(Pc, V, rS, vs); COL(Pp, V, rS, vsp);
            COL(Pc, W, rC, w0); COL(Pp, W, rC, wp);
            COL(Pc, YU, rC, y0); COL(Pp, YU, rC, yp); COL(Pm, YU, rC, ym); COL(Pc, YU, rN, yn); COL(Pc, YU, rS, ys);
            COL(Pp, YV, rC, zp); COL(Pp, YV, rS, zps); COL(Pc, YV, rC, z0); COL(Pc, YV, rS, zs);
            COL(Pc, YW, rC, q0); COL(Pp, YW, rC, qp);
#pragma unroll
            for (int m = 0; m < KV; m++) {
                const int a = m + 1;
                TC s = tcx * (yp[a] * (u0[a] + up[a]) - ym[a] * (um[a] + u0[a]));
                s = s + tcy * (yn[a] * (v0[a] + vp[a]) - ys[a] * (vs[a] + vsp[a]));
                s = s + c1[a + 1] * y0[a + 1] * (w0[a] + wp[a]);
                s = s - c2[a - 1] * y0[a - 1] * (w0[a - 1] + wp[a - 1]);
                s = s + tcx * (yp[a] * u0[a] + y0[a] * um[a] - y0[a] * up[a] - ym[a] * u0[a]);
                s = s + tcx * (zp[a] * v0[a] + zps[a] * vs[a] - z0[a] * vp[a] - zs[a] * vsp[a]);
                s = s + tcx * (qp[a] * w0[a] + qp[a - 1] * w0[a - 1] - q0[a] * wp[a] - q0[a - 1] * wp[a - 1]);
                ru[m] = (TOut)(alpha * s + (add_y ? y0[a] : TC(0)));
            }
        }
        {   // ---------------- gv ----------------
            TC u0[KV + 2], un[KV + 2], um[KV + 2], unm[KV + 2], v0[KV + 2], vn[KV + 2], vs[KV + 2];
            TC w0[KV + 2], wn[KV + 2], z0[KV + 2], zp[KV + 2], zm[KV + 2], zn[KV + 2], zs[KV + 2];
            TC yn[KV + 2], ynm[KV + 2], y0[KV + 2], ym[KV + 2], q0[KV + 2], qn[KV + 2];
            COL(Pc, U, rC, u0); COL(Pc, U, rN, un); COL(Pm, U, rC, um); COL(Pm, U, rN, unm);
            COL(Pc, V, rC, v0); COL(Pc, V, rN, vn); COL(Pc, V, rS, vs);
            COL(Pc, W, rC, w0); COL(Pc, W, rN, wn);
            COL(Pc, YV, rC, z0); COL(Pp, YV, rC, zp); COL(Pm, YV, rC, zm); COL(Pc, YV, rN, zn); COL(Pc, YV, rS, zs);
            COL(Pc, YU, rN, yn); COL(Pm, YU, rN, ynm); COL(Pc, YU, rC, y0); COL(Pm, YU, rC, ym);
            COL(Pc, YW, rC, q0); COL(Pc, YW, rN, qn);
#pragma unroll
            for (int m = 0; m < KV; m++) {
                const int a = m + 1;
                TC s = tcx * (zp[a] * (u0[a] + un[a]) - zm[a] * (um[a] + unm[a]));
                s = s + tcy * (zn[a] * (v0[a] + vn[a]) - zs[a] * (vs[a] + v0[a]));
                s = s + c1[a + 1] * z0[a + 1] * (w0[a] + wn[a]);
                s = s - c2[a - 1] * z0[a - 1] * (w0[a - 1] + wn[a - 1]);
                s = s + tcy * (yn[a] * u0[a] + ynm[a] * um[a] - y0[a] * un[a] - ym[a] * unm[a]);
                s = s + tcy * (zn[a] * v0[a] + z0[a] * vs[a] - z0[a] * vn[a] - zs[a] * v0[a]);
                s = s + tcy * (qn[a] * w0[a] + qn[a - 1] * w0[a - 1] - q0[a] * wn[a] - q0[a - 1] * wn[a - 1]);
                rv[m] = (TOut)(alpha * s + (add_y ? z0[a] : TC(0)));
            }
        }
        {   // ---------------- gw ----------------
            TC u0[KV + 2], um[KV + 2], v0[KV + 2], vs[KV + 2], w0[KV + 2];
            TC q0[KV + 2], qp[KV + 2], qm[KV + 2], qn[KV + 2], qs[KV + 2];
            TC y0[KV + 2], ym[KV + 2], z0[KV + 2], zs[KV + 2];
            COL(Pc, U, rC, u0); COL(Pm, U, rC, um); COL(Pc, V, rC, v0); COL(Pc, V, rS, vs);
            COL(Pc, W, rC, w0);
            COL(Pc, YW, rC, q0); COL(Pp, YW, rC, qp); COL(Pm, YW, rC, qm); COL(Pc, YW, rN, qn); COL(Pc, YW, rS, qs);
            COL(Pc, YU, rC, y0); COL(Pm, YU, rC, ym); COL(Pc, YV, rC, z0); COL(Pc, YV, rS, zs);
#pragma unroll
            for (int m = 0; m < KV; m++) {
                const int a = m + 1;
                TC s = tcx * (qp[a] * (u0[a] + u0[a + 1]) - qm[a] * (um[a] + um[a + 1]));
                s = s + tcy * (qn[a] * (v0[a] + v0[a + 1]) - qs[a] * (vs[a] + vs[a + 1]));
                s = s + d1[a + 1] * q0[a + 1] * (w0[a] + w0[a + 1]);
                s = s - d2[a - 1] * q0[a - 1] * (w0[a - 1] + w0[a]);
                s = s + c1[a + 1] * (y0[a + 1] * u0[a] + ym[a + 1] * um[a]);
                s = s - c2[a] * (y0[a] * u0[a + 1] + ym[a] * um[a + 1]);
                s = s + c1[a + 1] * (z0[a + 1] * v0[a] + zs[a + 1] * vs[a]);
                s = s - c2[a] * (z0[a] * v0[a + 1] + zs[a] * vs[a + 1]);
                s = s + d1[a + 1] * q0[a + 1] * w0[a] + d1[a] * q0[a] * w0[a - 1];
                s = s - d2[a] * q0[a] * w0[a + 1] - d2[a - 1] * q0[a - 1] * w0[a];
                rw[m] = (kbase + m < nzl) ? (TOut)(alpha * s + (add_y ? q0[a] : TC(0))) : TOut(0);
            }
        }
#undef COL
        if (active) {
            const long long off = (long long)(i + 2) * g.si + (long long)(j + 2) * g.sj + kbase;
            pw_store<TOut, KV>(gu + off, ru, nvalid, beta);
            pw_store<TOut, KV>(gv + off, rv, nvalid, beta);
            pw_store<TOut, KV>(gw + off, rw, nvalid, beta);
        }
    }
}

template <typename TS, typename TC, int KV>
static pw_status pw_launch_adjoint(const pw_mesh *m, const void *const *in, void *const *out,
                                   double alpha, int beta, int add_y, cudaStream_t st, int tile_j,
                                   int tile_i, int ns) {
    PwAdjGeom g;
    g.nx = m->nx;
    g.ny = m->ny;
    g.nz = m->nz;
    g.nzp = m->nzp;
    g.h = 16 / (int)sizeof(TS);
    int unit = KV > g.h ? KV : g.h;
    int kc_one = (m->nz + unit - 1) / unit * unit;
    g.kc = (kc_one + 2 * g.h <= 256) ? kc_one : 128;
    g.kb = g.kc + 2 * g.h;
    // rows per CTA: as asked, but no more than 256 threads (long columns)
    tile_j = tile_j < 256 / (g.kc / KV) ? tile_j : 256 / (g.kc / KV);
    if (tile_j < 1) tile_j = 1;
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
    int threads = (g.kc / KV) * tile_j;
    if (threads > 256) return pw_fail(PW_ERR_SHAPE, "adjoint tile needs %d threads", threads);
    size_t smem = (size_t)ns * 6 * g.field_stride * sizeof(TS) + (size_t)ns * sizeof(uint64_t);
    if (smem > 226 * 1024) return pw_fail(PW_ERR_SHAPE, "adjoint tile needs %zu bytes of shared memory", smem);
    CUtensorMap maps[6];
    for (int q = 0; q < 6; q++) {
        pw_status s = pw_make_field_map(&maps[q], in[q], m->dtype, m->nx, m->ny, m->nzp, pw_kdim(m->nz, q % 3),
                                        g.kb, tile_j + 2);
        if (s != PW_OK) return s;
    }
    auto kern = pw_adjoint_march<TS, TC, KV>;
    PW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // a CTA marches ti columns from ti + 2 planes
    tile_i = pw_pick_tile_i(m, tile_i, tiles, pw_slots(m, kern, threads, smem), 2);
    g.ti = tile_i;
    dim3 grid((unsigned)((m->ny + tile_j - 1) / tile_j), (unsigned)((m->nx + tile_i - 1) / tile_i),
              (unsigned)((m->nz + g.kc - 1) / g.kc));
    if (grid.y > 65535 || grid.z > 65535) return pw_fail(PW_ERR_SHAPE, "grid too large");
    const TC *coef = std::is_same<TC, double>::value
                         ? reinterpret_cast<const TC *>(m->coef64 + 6 * m->nz)
                         : reinterpret_cast<const TC *>(m->coef32);
    kern<<<grid, threads, smem, st>>>(maps[0], maps[1], maps[2], maps[3], maps[4], maps[5],
                                      (TS *)out[0], (TS *)out[1], (TS *)out[2], coef, g, (TC)alpha, beta,
                                      add_y, m->status);
    PW_CUDA(cudaGetLastError());
    return PW_OK;
}

static pw_status pw_adjoint_common(const pw_mesh *m, const void *u, const void *v, const void *w,
                                   void *gsu, void *gsv, void *gsw, void *gu, void *gv, void *gw,
                                   double alpha, int beta, int add_y, void *stream) {
    if (!m) return pw_fail(PW_ERR_ARG, "mesh is NULL");
    if (beta != 0 && beta != 1) return pw_fail(PW_ERR_ARG, "beta must be 0 or 1");
    if (!isfinite(alpha)) return pw_fail(PW_ERR_ARG, "alpha/dt must be finite");
    const void *p[9] = {u, v, w, gsu, gsv, gsw, gu, gv, gw};
    const char *nm[9] = {"u", "v", "w", "gsu", "gsv", "gsw", "gu", "gv", "gw"};
    for (int q = 0; q < 9; q++) {
        pw_status s = pw_check_ptr(p[q], nm[q]);
        if (s != PW_OK) return s;
    }
    for (int a = 0; a < 6; a++)
        for (int b = 6; b < 9; b++)
            if (p[a] == p[b]) return pw_fail(PW_ERR_ARG, "%s and %s alias", nm[a], nm[b]);
    if (m->dtype != PW_F32 && m->dtype != PW_F64)
        return pw_fail(PW_ERR_DTYPE, "the adjoint is available for PW_F32 and PW_F64 meshes");
    cudaStream_t st = (cudaStream_t)stream;
    if (m->nz == 1) {  // sw is identically 0 and w is all lid: gsw carries nothing
        const size_t bytes = (size_t)m->total * pw_elem_in(m->dtype);
        PW_CUDA(cudaMemsetAsync(gsw, 0, bytes, st));
    }
    void *ys[3] = {gsu, gsv, gsw};
    pw_status s = pw_launch_halo(m, ys, 3, st);
    if (s != PW_OK) return s;
    const void *in[6] = {u, v, w, gsu, gsv, gsw};
    void *out[3] = {gu, gv, gw};
    if (m->dtype == PW_F32)
        return pw_launch_adjoint<float, float, 2>(m, in, out, alpha, beta, add_y, st, 4, m->tile_i, 4);
    if (m->algo == PW_ALGO_F64_SPLIT) return pw_launch_adjoint_split(m, in, out, alpha, beta, add_y, st);
    return pw_launch_adjoint<double, double, 2>(m, in, out, alpha, beta, add_y, st, 4, m->tile_i, 4);
}

extern "C" pw_status pw_advect_adjoint(const pw_mesh *m, const void *u, const void *v, const void *w,
                                       void *gsu, void *gsv, void *gsw, void *gu, void *gv, void *gw,
                                       double alpha, int beta, void *stream) {
    return pw_adjoint_common(m, u, v, w, gsu, gsv, gsw, gu, gv, gw, alpha, beta, 0, stream);
}

extern "C" pw_status pw_euler_adjoint(const pw_mesh *m, const void *u, const void *v, const void *w,
                                      void *gu_in, void *gv_in, void *gw_in, void *gu_out,
                                      void *gv_out, void *gw_out, double dt, void *stream) {
    return pw_adjoint_common(m, u, v, w, gu_in, gv_in, gw_in, gu_out, gv_out, gw_out, dt, 0, 1,
                             stream);
}
