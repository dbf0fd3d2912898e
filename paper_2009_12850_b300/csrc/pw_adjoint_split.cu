// pw_adjoint_split.cu -- the adjoint of the PW stencil for FP64 meshes in
// double-float arithmetic on the FP32 pipe (the default FP64 path, as for the
// forward stencil): gu, gv, gw = alpha J(u,v,w)^T (gsu, gsv, gsw) [+ g_in].
//
// The gather form of pw_adjoint.cu (every forward product is differentiated
// from the receiving point's side) written in the split arithmetic of
// pw_advect_split.cu: six fields (u, v, w and the incoming gradients y, z, q)
// are staged per x plane by TMA, converted with integer bit operations into
// (hi, hi, lo, lo) chunks that pair levels k and k + KC/2, and each thread
// computes its row at those two levels with packed .f32x2 double-float
// products and sums; each output is rebuilt with one FP64 add.  Fields and
// gradients are carried scaled by 2^8, products by 2^16 (removed by the join);
// the term g_in of the Euler adjoint is added in FP64 from the exact value in
// memory.  Vertical coefficients are the products tzc1, tzc2, tzd1, tzd2, split
// unscaled into float pairs.
#include <math.h>

#include "pw_df.cuh"
#include "pw_internal.h"

struct PwAdjSplitGeom {
    int nx, ny, nz;
    int kc, half, ti;
    int rfs;  // doubles between the six planes of a raw slot (128-byte aligned)
    long long si, sj;
    double tcx, tcy;
};

// one raw TMA slot and three converted planes (i-1, i, i+1): 72 KB, so three
// CTAs share an SM; converting into the slot of plane i-2 needs a barrier after
// the previous step, and the raw slot is refilled after a second barrier
#define PW_ASPLIT_RAW 1
#define PW_ASPLIT_CONV 3

__device__ __forceinline__ D2 pw_ald(const float4 *p, int q) {
    const float4 c = p[q];
    return D2{pk(c.x, c.y), pk(c.z, c.w)};
}

// unscaled float pair of a double coefficient (hi = nearest float, lo = rest)
__device__ __forceinline__ float2 pw_coef_pair(double c) {
    const float h = (float)c;
    return make_float2(h, (float)(c - (double)h));
}

template <int TJ, int KC, bool ISO>
__global__ void __launch_bounds__(TJ *(KC > 0 ? KC / 2 : (TJ == 4 ? 32 : 16)), 3)
pw_adjoint_split_kernel(const __grid_constant__ CUtensorMap mu, const __grid_constant__ CUtensorMap mv,
                        const __grid_constant__ CUtensorMap mw, const __grid_constant__ CUtensorMap my,
                        const __grid_constant__ CUtensorMap mz, const __grid_constant__ CUtensorMap mq,
                        double *__restrict__ gu, double *__restrict__ gv, double *__restrict__ gw,
                        const double *__restrict__ yu, const double *__restrict__ yv,
                        const double *__restrict__ yw, const double *__restrict__ coef,
                        const PwAdjSplitGeom g, double alpha, int beta, int add_y,
                        int *__restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int NF = 6;
    constexpr int ROWS = NF * (TJ + 2);
    constexpr bool CT = KC > 0;
    constexpr int RFS_CT = CT ? ((TJ + 2) * (KC + 4) + 15) / 16 * 16 : 0;
    const int half = CT ? KC / 2 : g.half;
    const int cw = half + 2, kb = 2 * half + 4;
    const int rfs = CT ? RFS_CT : g.rfs;
    const int cfs = (TJ + 2) * cw;
    const int nt = CT ? (KC / 2) * TJ : (int)blockDim.x;
    double *raw = reinterpret_cast<double *>(smem_raw);
    float4 *conv = reinterpret_cast<float4 *>(smem_raw + (size_t)PW_ASPLIT_RAW * NF * rfs * 8);
    uint64_t *bars = reinterpret_cast<uint64_t *>(conv + (size_t)PW_ASPLIT_CONV * NF * cfs);
    float4 *ctab = reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(bars) + 64);
    const int tid = threadIdx.x;
    const int tk = tid % half, tj = tid / half;
    const int j0 = blockIdx.y * TJ, i0 = blockIdx.z * g.ti, k0 = blockIdx.x * 2 * half;
    const int i_end = min(i0 + g.ti, g.nx);
    const int nplanes = i_end - i0 + 2;
    const uint32_t plane_bytes = (uint32_t)NF * (uint32_t)(TJ + 2) * (uint32_t)kb * 8u;
    const int ka = k0 + tk, kz = ka + half;
    const int j = j0 + tj;
    const CUtensorMap *maps[NF] = {&mu, &mv, &mw, &my, &mz, &mq};

    if (pw_cta_failed(status)) return;
    if (tid == 0) {
        for (int f = 0; f < NF; f++) pw_prefetch_map(maps[f]);
        for (int s = 0; s < PW_ASPLIT_RAW; s++) pw_mbar_init(&bars[s], 1);
        pw_fence_barrier_init();
    }
    __syncthreads();
    auto issue = [&](int p) {
        const int s = p % PW_ASPLIT_RAW;
        double *dst = raw + (size_t)s * NF * rfs;
        pw_mbar_expect_tx(&bars[s], plane_bytes);
        const int c0 = k0 - 2, c1 = j0 + 1, c2 = i0 + 1 + p;
#pragma unroll
        for (int f = 0; f < NF; f++) pw_tma_load_3d(dst + (size_t)f * rfs, maps[f], c0, c1, c2, &bars[s]);
    };
    int issued = 0;
    if (tid == 0) {
        for (int p = 0; p < min(PW_ASPLIT_RAW, nplanes); p++) issue(p);
        issued = min(PW_ASPLIT_RAW, nplanes);
    }
    auto give_up = [&](int from) {
        if (tid == 0) {
            for (int p = from; p < issued; p++)
                if (!pw_mbar_wait_bounded(&bars[p % PW_ASPLIT_RAW], (uint32_t)((p / PW_ASPLIT_RAW) & 1),
                                          PW_DRAIN_CYCLES))
                    break;
            atomicExch(status, (int)PW_ERR_TIMEOUT);
        }
    };

    // conversion of raw plane p into converted slot p % PW_ASPLIT_CONV (chunk
    // q of a row: levels k0+q-1 and k0+q-1+half)
    bool bad = false;
    constexpr int MR = (ROWS + TJ - 1) / TJ;
    auto src_of = [&](int R, int q) {
        const int f = R / (TJ + 2);
        return f * rfs + (R - f * (TJ + 2)) * kb + q + 1;
    };
    auto conv_one = [&](const double *rs, float4 *cd, int so, int dof) {
        const uint2 a = *reinterpret_cast<const uint2 *>(rs + so);
        const uint2 b = *reinterpret_cast<const uint2 *>(rs + so + half);
        float ha, la, hb, lb;
        split_words(a.x, a.y, ha, la, PW_SPLIT_WIND_EHI, bad);
        split_words(b.x, b.y, hb, lb, PW_SPLIT_WIND_EHI, bad);
        cd[dof] = make_float4(ha, hb, la, lb);
    };
    auto convert = [&](int p) {
        const double *rs = raw + (size_t)(p % PW_ASPLIT_RAW) * NF * rfs;
        float4 *cd = conv + (size_t)(p % PW_ASPLIT_CONV) * NF * cfs;
#pragma unroll
        for (int m = 0; m < MR; m++) {
            const int R = tj + m * TJ;
            if (R < ROWS) conv_one(rs, cd, src_of(R, tk + 1), R * cw + tk + 1);
        }
        for (int e = tid; e < 2 * ROWS; e += nt) {
            const int R = e >> 1, q = (e & 1) ? cw - 1 : 0;
            conv_one(rs, cd, src_of(R, q), R * cw + q);
        }
        pw_fence_proxy_async();
    };

    // vertical coefficients of this thread's level pair (ka, kz), split into
    // float pairs once per CTA: C1p = tzc1(k+1), C2m = tzc2(k-1), C2 = tzc2(k),
    // D1p = tzd1(k+1), D1 = tzd1(k), D2 = tzd2(k), D2m = tzd2(k-1); 0 outside
    // the grid (tzd is 0 on the lid face already)
    auto cget = [&](int arr, int k) { return (k >= 0 && k < g.nz) ? coef[arr * g.nz + k] : 0.0; };
    for (int t = tid; t < half; t += nt) {
        const int a = k0 + t, b = a + half;
        const int arrs[7] = {0, 1, 1, 2, 2, 3, 3};
        const int offs[7] = {1, -1, 0, 1, 0, 0, -1};
        for (int c = 0; c < 7; c++) {
            const float2 x = pw_coef_pair(cget(arrs[c], a + offs[c]));
            const float2 y = pw_coef_pair(cget(arrs[c], b + offs[c]));
            ctab[t * 7 + c] = make_float4(x.x, y.x, x.y, y.y);
        }
    }
    if (tid == 0) {
        const float2 x = pw_coef_pair(g.tcx), y = pw_coef_pair(g.tcy);
        ctab[half * 7] = make_float4(x.x, x.x, x.y, x.y);
        ctab[half * 7 + 1] = make_float4(y.x, y.x, y.y, y.y);
    }
    const bool active = j < g.ny;
    const bool oka = ka < g.nz, okz = kz < g.nz;
    const int tb = tj * cw + tk + 1;
    auto base = [&](int p) { return conv + (size_t)(p % PW_ASPLIT_CONV) * NF * cfs + tb; };
    // field f (0 u, 1 v, 2 w, 3 y = gsu, 4 z = gsv, 5 q = gsw), row o (0: j-1, 1: j, 2: j+1), shift sh
    auto L = [&](const float4 *B, int f, int o, int sh) { return pw_ald(B, f * cfs + o * cw + sh); };

    for (int p = 0; p < nplanes; p++) {
        // the raw plane p has landed and every thread is past step p-1 (its
        // converted slot, that of plane p-3, is free)
        const bool ok = pw_mbar_wait_bounded(&bars[p % PW_ASPLIT_RAW], (uint32_t)((p / PW_ASPLIT_RAW) & 1));
        if (!__syncthreads_and(ok)) {
            give_up(p);
            return;
        }
        convert(p);
        __syncthreads();  // plane p converted; the raw slot takes plane p + 1
        if (tid == 0 && p + PW_ASPLIT_RAW < nplanes) {
            issue(p + PW_ASPLIT_RAW);
            issued = p + PW_ASPLIT_RAW + 1;
        }
        if (p < 2) continue;
        const int i = i0 + p - 2;
        const float4 *BM = base(p - 2), *BC = base(p - 1), *BP = base(p);
        const D2 tcx = pw_ald(ctab, half * 7), tcy = pw_ald(ctab, half * 7 + 1);
        // tcx X + tcy Y + Z; with tcx == tcy (a square horizontal grid) one product
        auto horiz = [&](D2 X, D2 Y, D2 Z) {
            if constexpr (ISO) return df_add(df_mul(tcx, df_add(X, Y)), Z);
            else return df_add(df_add(df_mul(tcx, X), df_mul(tcy, Y)), Z);
        };
        const float4 *ct = ctab + tk * 7;
        const D2 C1p = pw_ald(ct, 0), C2m = pw_ald(ct, 1), C2 = pw_ald(ct, 2);
        const D2 D1p = pw_ald(ct, 3), D1 = pw_ald(ct, 4), Dd2 = pw_ald(ct, 5), D2m = pw_ald(ct, 6);
        enum { U = 0, V = 1, W = 2, Y = 3, Z = 4, Q = 5 };

        // ---------------- gu ----------------
        D2 ru;
        {
            const D2 u0 = L(BC, U, 1, 0), up = L(BP, U, 1, 0), um = L(BM, U, 1, 0);
            const D2 v0 = L(BC, V, 1, 0), vp = L(BP, V, 1, 0), vs = L(BC, V, 0, 0), vsp = L(BP, V, 0, 0);
            const D2 w0 = L(BC, W, 1, 0), wp = L(BP, W, 1, 0), w0m = L(BC, W, 1, -1), wpm = L(BP, W, 1, -1);
            const D2 y0 = L(BC, Y, 1, 0), yp = L(BP, Y, 1, 0), ym = L(BM, Y, 1, 0);
            const D2 yn = L(BC, Y, 2, 0), ys = L(BC, Y, 0, 0), y0p = L(BC, Y, 1, 1), y0m = L(BC, Y, 1, -1);
            const D2 zp = L(BP, Z, 1, 0), zps = L(BP, Z, 0, 0), z0 = L(BC, Z, 1, 0), zs = L(BC, Z, 0, 0);
            const D2 q0 = L(BC, Q, 1, 0), qp = L(BP, Q, 1, 0), q0m = L(BC, Q, 1, -1), qpm = L(BP, Q, 1, -1);
            // x: advected u and its advecting u, v, w faces
            D2 X = df_sub(df_mul(yp, df_add(u0, up)), df_mul(ym, df_add(um, u0)));
            X = df_add(X, df_sub(df_mul(u0, df_sub(yp, ym)), df_mul(y0, df_sub(up, um))));
            X = df_add(X, df_sub(df_add(df_mul(zp, v0), df_mul(zps, vs)), df_add(df_mul(z0, vp), df_mul(zs, vsp))));
            X = df_add(X, df_sub(df_add(df_mul(qp, w0), df_mul(qpm, w0m)), df_add(df_mul(q0, wp), df_mul(q0m, wpm))));
            const D2 Yt = df_sub(df_mul(yn, df_add(v0, vp)), df_mul(ys, df_add(vs, vsp)));
            const D2 Zt = df_sub(df_mul(df_mul(C1p, y0p), df_add(w0, wp)), df_mul(df_mul(C2m, y0m), df_add(w0m, wpm)));
            ru = horiz(X, Yt, Zt);
        }
        // ---------------- gv ----------------
        D2 rv;
        {
            const D2 u0 = L(BC, U, 1, 0), un = L(BC, U, 2, 0), um = L(BM, U, 1, 0), unm = L(BM, U, 2, 0);
            const D2 v0 = L(BC, V, 1, 0), vn = L(BC, V, 2, 0), vs = L(BC, V, 0, 0);
            const D2 w0 = L(BC, W, 1, 0), wn = L(BC, W, 2, 0), w0m = L(BC, W, 1, -1), wnm = L(BC, W, 2, -1);
            const D2 z0 = L(BC, Z, 1, 0), zp = L(BP, Z, 1, 0), zm = L(BM, Z, 1, 0), zn = L(BC, Z, 2, 0);
            const D2 zs = L(BC, Z, 0, 0), z0p = L(BC, Z, 1, 1), z0m = L(BC, Z, 1, -1);
            const D2 yn = L(BC, Y, 2, 0), ynm = L(BM, Y, 2, 0), y0 = L(BC, Y, 1, 0), ym = L(BM, Y, 1, 0);
            const D2 q0 = L(BC, Q, 1, 0), qn = L(BC, Q, 2, 0), q0m = L(BC, Q, 1, -1), qnm = L(BC, Q, 2, -1);
            const D2 Xt = df_sub(df_mul(zp, df_add(u0, un)), df_mul(zm, df_add(um, unm)));
            // y: advected v and its advecting u, v, w faces
            D2 Yt = df_sub(df_mul(zn, df_add(v0, vn)), df_mul(zs, df_add(vs, v0)));
            Yt = df_add(Yt, df_sub(df_add(df_mul(yn, u0), df_mul(ynm, um)), df_add(df_mul(y0, un), df_mul(ym, unm))));
            Yt = df_add(Yt, df_sub(df_mul(v0, df_sub(zn, zs)), df_mul(z0, df_sub(vn, vs))));
            Yt = df_add(Yt, df_sub(df_add(df_mul(qn, w0), df_mul(qnm, w0m)), df_add(df_mul(q0, wn), df_mul(q0m, wnm))));
            const D2 Zt = df_sub(df_mul(df_mul(C1p, z0p), df_add(w0, wn)), df_mul(df_mul(C2m, z0m), df_add(w0m, wnm)));
            rv = horiz(Xt, Yt, Zt);
        }
        // ---------------- gw ----------------
        D2 rw;
        {
            const D2 u0 = L(BC, U, 1, 0), um = L(BM, U, 1, 0), u0p = L(BC, U, 1, 1), ump = L(BM, U, 1, 1);
            const D2 v0 = L(BC, V, 1, 0), vs = L(BC, V, 0, 0), v0p = L(BC, V, 1, 1), vsp = L(BC, V, 0, 1);
            const D2 w0 = L(BC, W, 1, 0), w0p = L(BC, W, 1, 1), w0m = L(BC, W, 1, -1);
            const D2 q0 = L(BC, Q, 1, 0), qp = L(BP, Q, 1, 0), qm = L(BM, Q, 1, 0), qn = L(BC, Q, 2, 0);
            const D2 qs = L(BC, Q, 0, 0), q0p = L(BC, Q, 1, 1), q0m = L(BC, Q, 1, -1);
            const D2 y0 = L(BC, Y, 1, 0), ym = L(BM, Y, 1, 0), y0p = L(BC, Y, 1, 1), ymp = L(BM, Y, 1, 1);
            const D2 z0 = L(BC, Z, 1, 0), zs = L(BC, Z, 0, 0), z0p = L(BC, Z, 1, 1), zsp = L(BC, Z, 0, 1);
            const D2 Xt = df_sub(df_mul(qp, df_add(u0, u0p)), df_mul(qm, df_add(um, ump)));
            const D2 Yt = df_sub(df_mul(qn, df_add(v0, v0p)), df_mul(qs, df_add(vs, vsp)));
            // z: advected w and its advecting w faces, and the w faces of u and v
            D2 Zt = df_sub(df_mul(df_mul(D1p, q0p), df_add(w0, w0p)), df_mul(df_mul(D2m, q0m), df_add(w0m, w0)));
            Zt = df_add(Zt, df_mul(C1p, df_add(df_mul(y0p, u0), df_mul(ymp, um))));
            Zt = df_sub(Zt, df_mul(C2, df_add(df_mul(y0, u0p), df_mul(ym, ump))));
            Zt = df_add(Zt, df_mul(C1p, df_add(df_mul(z0p, v0), df_mul(zsp, vs))));
            Zt = df_sub(Zt, df_mul(C2, df_add(df_mul(z0, v0p), df_mul(zs, vsp))));
            Zt = df_add(Zt, df_add(df_mul(df_mul(D1p, q0p), w0), df_mul(df_mul(D1, q0), w0m)));
            Zt = df_sub(Zt, df_add(df_mul(df_mul(Dd2, q0), w0p), df_mul(df_mul(D2m, q0m), w0)));
            rw = horiz(Xt, Yt, Zt);
        }
        if (!active) continue;

        // ---------------- outputs: levels ka and kz ----------------
        const long long off = (long long)(i + 2) * g.si + (long long)(j + 2) * g.sj;
        const double ga[3] = {join(lx(ru.h), lx(ru.l)), join(lx(rv.h), lx(rv.l)), join(lx(rw.h), lx(rw.l))};
        const double gz[3] = {join(ly(ru.h), ly(ru.l)), join(ly(rv.h), ly(rv.l)), join(ly(rw.h), ly(rw.l))};
        double *outs[3] = {gu, gv, gw};
        const double *ins[3] = {yu, yv, yw};
#pragma unroll
        for (int c = 0; c < 3; c++) {
            if (oka) {
                const long long o = off + ka;
                double r = alpha * ga[c] + (add_y ? ins[c][o] : 0.0);
                if (c == 2 && ka >= g.nz - 1) r = 0.0;  // the lid face is not a degree of freedom
                outs[c][o] = beta ? outs[c][o] + r : r;
            }
            if (okz) {
                const long long o = off + kz;
                double r = alpha * gz[c] + (add_y ? ins[c][o] : 0.0);
                if (c == 2 && kz >= g.nz - 1) r = 0.0;
                outs[c][o] = beta ? outs[c][o] + r : r;
            }
        }
    }
    if (__syncthreads_or(bad) && tid == 0) atomicOr(status + PW_STATUS_RANGE_WORD, 1);
}

pw_status pw_launch_adjoint_split(const pw_mesh *m, const void *const *in, void *const *out, double alpha,
                                  int beta, int add_y, cudaStream_t st) {
    const int tile_j = 8, kc_max = 32;
    PwAdjSplitGeom g;
    g.nx = m->nx;
    g.ny = m->ny;
    g.nz = m->nz;
    const int kc_one = (m->nz + 1) / 2 * 2;
    g.kc = kc_one <= kc_max ? kc_one : kc_max;
    g.half = g.kc / 2;
    const int kb = g.kc + 4, cw = g.half + 2;
    const long tiles = (long)((m->ny + tile_j - 1) / tile_j) * ((m->nz + g.kc - 1) / g.kc);
    g.rfs = ((tile_j + 2) * kb + 15) / 16 * 16;
    g.si = m->si;
    g.sj = m->sj;
    g.tcx = m->tcx;
    g.tcy = m->tcy;
    const int threads = g.half * tile_j;
    const size_t smem = (size_t)PW_ASPLIT_RAW * 6 * g.rfs * 8 + (size_t)PW_ASPLIT_CONV * 6 * (tile_j + 2) * cw * 16 +
                        64 + ((size_t)g.half * 7 + 2) * sizeof(float4);
    if (smem > 226 * 1024) return pw_fail(PW_ERR_SHAPE, "split adjoint needs %zu bytes of shared memory", smem);
    CUtensorMap maps[6];
    for (int q = 0; q < 6; q++) {
        pw_status s = pw_make_field_map(&maps[q], in[q], PW_F64, m->nx, m->ny, m->nzp, pw_kdim(m->nz, q % 3), kb,
                                        tile_j + 2);
        if (s != PW_OK) return s;
    }
    const bool iso = m->tcx == m->tcy;
    auto kern = g.kc == kc_max ? (iso ? pw_adjoint_split_kernel<8, 32, true> : pw_adjoint_split_kernel<8, 32, false>)
                               : (iso ? pw_adjoint_split_kernel<8, 0, true> : pw_adjoint_split_kernel<8, 0, false>);
    PW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // a CTA marches ti columns from ti + 2 planes
    g.ti = pw_pick_tile_i(m, m->tile_i, tiles, pw_slots(m, kern, threads, smem), 2);
    dim3 grid((unsigned)((m->nz + g.kc - 1) / g.kc), (unsigned)((m->ny + tile_j - 1) / tile_j),
              (unsigned)((m->nx + g.ti - 1) / g.ti));
    if (grid.y > 65535 || grid.z > 65535) return pw_fail(PW_ERR_SHAPE, "grid too large");
    kern<<<grid, threads, smem, st>>>(maps[0], maps[1], maps[2], maps[3], maps[4], maps[5], (double *)out[0],
                                      (double *)out[1], (double *)out[2], (const double *)in[3],
                                      (const double *)in[4], (const double *)in[5], m->coef64 + 6 * m->nz, g,
                                      alpha, beta, add_y, m->status);
    PW_CUDA(cudaGetLastError());
    return PW_OK;
}
