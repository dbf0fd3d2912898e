// pw_advect_split.cu -- FP64 PW stencil in double-float arithmetic (FP64 in,
// FP64 out, error within a few units of 2^-46 of the per-point condition sum).
//
// Why: B300's FP64 units run at ~1.6 operations / clock / SM, so native FP64
// caps this ~42-FLOP-per-point stencil near 11 Gpoints/s (8% of the HBM
// roofline).  Here every double is split exactly-enough into two floats and the
// stencil runs on the FP32 pipe (packed .f32x2 instructions over two k levels),
// with FP64 used only for one add per output.
//
// Layout of the work: the same x-march as the FP32 kernel.  A CTA of 128 threads
// owns tile_j rows and a k chunk (8 rows x 32 levels by default, or 4 x 64); the
// k chunk is the fastest grid index, so the chunks of a column run together and
// the k-halo levels they share come from L2.  TMA brings (j,k) planes of u, v, w (doubles) into a ring
// of NS shared-memory slots (levels >= nz and the w lid arrive as zeros: the
// tensor maps carry the logical k extent); when a plane has landed, all threads
// convert it in place, 16 bytes at a time, from (x_k, x_k+1) to
// (hi_k, hi_k+1, lo_k, lo_k+1).  Each
// thread then computes two levels (k, k+1) of one column per step.
//
// The algebra is the PW form regrouped around the face coefficients:
//   tzc1(k) = g(k-1) r(k), tzc2(k) = g(k) r(k),   g = 0.25 rho_w, r = 1/(rho_n dz)
//   tzd1(k) = g'(k) r'(k), tzd2(k) = g'(k+1) r'(k), g' = 0.25 rho_n, r' = 1/(rho_w dzn)
// so that  s = tcx X + tcy Y + r Z  with X, Y, Z differences of products of a
// field value and an (unscaled, or g-scaled for the vertical) face sum.
#include <algorithm>

#include "pw_df.cuh"
#include "pw_internal.h"
#include "pw_march.cuh"  // pw_store_images

struct PwSplitGeom {
    int nx, ny, nz, kc, kb, tj, ti;
    int rows;          // 3 * (tj + 2) rows per plane (u, v, w)
    int cpr;           // 16-byte chunks per plane row = kb / 2
    float inv_cpr;
    int field_stride;  // doubles between the u, v, w planes of a slot
    int cs_n;          // levels in the coefficient table (nz + 4, level -2 first)
    long long si, sj;
};

// STEP: write x + dt S(x) (x read exactly from xu, xv, xw) to su, sv, sw and to
// their periodic halo images, the forward Euler step fused into the stencil
template <int NS, int TJ, bool BETA, bool STEP = false>
__global__ void __launch_bounds__(256, 2)
pw_advect_split_kernel(const __grid_constant__ CUtensorMap mu, const __grid_constant__ CUtensorMap mv,
                       const __grid_constant__ CUtensorMap mw, double *__restrict__ su,
                       double *__restrict__ sv, double *__restrict__ sw,
                       const float *__restrict__ cs, const PwSplitGeom g,
                       int *__restrict__ status, const double *__restrict__ xu = nullptr,
                       const double *__restrict__ xv = nullptr, const double *__restrict__ xw = nullptr,
                       double dt = 0.0) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    double *planes = reinterpret_cast<double *>(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + (size_t)NS * 3 * g.field_stride * 8);
    const int nt = blockDim.x, tid = threadIdx.x;
    const int nkt = g.kc / 2;
    const int tk = tid % nkt, tj = tid / nkt;
    // k chunks are the fastest grid index: the chunks of a column run together,
    // so the k-halo levels they share are fetched from DRAM once (L2 hits)
    const int j0 = blockIdx.y * TJ, i0 = blockIdx.z * g.ti, k0 = blockIdx.x * g.kc;
    const int i_end = min(i0 + g.ti, g.nx);
    const int nplanes = i_end - i0 + 2;
    const uint32_t plane_bytes = 3u * (uint32_t)(TJ + 2) * (uint32_t)g.kb * 8u;
    const int kbase = k0 + 2 * tk, kk = 2 + 2 * tk, j = j0 + tj;
    const int fs = g.field_stride;

    if (pw_cta_failed(status)) return;
    if (tid == 0) {
        pw_prefetch_map(&mu);
        pw_prefetch_map(&mv);
        pw_prefetch_map(&mw);
        for (int s = 0; s < NS; s++) pw_mbar_init(&bars[s], 1);
        pw_fence_barrier_init();
    }
    __syncthreads();
    auto issue = [&](int p) {
        const int s = p % NS;
        double *dst = planes + (size_t)s * 3 * fs;
        pw_mbar_expect_tx(&bars[s], plane_bytes);
        const int c0 = k0 - 2, c1 = j0 + 1, c2 = i0 + 1 + p;
        pw_tma_load_3d(dst, &mu, c0, c1, c2, &bars[s]);
        pw_tma_load_3d(dst + fs, &mv, c0, c1, c2, &bars[s]);
        pw_tma_load_3d(dst + 2 * fs, &mw, c0, c1, c2, &bars[s]);
    };
    int issued = 0;
    if (tid == 0) {
        for (int p = 0; p < min(NS, nplanes); p++) issue(p);
        issued = min(NS, nplanes);
    }
    auto wait = [&](int p) {
        return pw_mbar_wait_bounded(&bars[p % NS], (uint32_t)((p / NS) & 1));
    };
    auto give_up = [&](int from) {
        if (tid == 0) {
            for (int p = from; p < issued; p++)
                if (!pw_mbar_wait_bounded(&bars[p % NS], (uint32_t)((p / NS) & 1), PW_DRAIN_CYCLES)) break;
            atomicExch(status, (int)PW_ERR_TIMEOUT);
        }
    };
    // in-place conversion of a landed plane: doubles -> (hi, hi, lo, lo) chunks.
    // Thread (tk, tj) converts chunk tk+1 of rows tj, tj+TJ, ... of the
    // 3*(TJ+2) rows (u, v, w); the first 6*(TJ+2) threads also convert one of
    // the two edge chunks (k halo) of a row.
    constexpr int ROWS = 3 * (TJ + 2);
    bool bad = false;  // a value this thread converted was outside the split range
    auto conv_chunk = [&](double *base, int R, int q) {
        const int f = R / (TJ + 2), r = R - f * (TJ + 2);
        double *cp = base + (size_t)f * fs + (size_t)r * g.kb + 2 * q;
        // (lo, hi) words of two doubles; levels >= nz and the w lid arrived as 0
        const uint4 d = *reinterpret_cast<const uint4 *>(cp);
        float h0, l0, h1, l1;
        split_words(d.x, d.y, h0, l0, PW_SPLIT_WIND_EHI, bad);
        split_words(d.z, d.w, h1, l1, PW_SPLIT_WIND_EHI, bad);
        *reinterpret_cast<float4 *>(cp) = make_float4(h0, h1, l0, l1);
    };
    auto convert = [&](int p) {
        double *base = planes + (size_t)(p % NS) * 3 * fs;
#pragma unroll
        for (int m = 0; m < (ROWS + TJ - 1) / TJ; m++) {
            const int R = tj + m * TJ;
            if (R < ROWS) conv_chunk(base, R, tk + 1);
        }
        for (int e = tid; e < 2 * ROWS; e += nt) conv_chunk(base, e >> 1, (e & 1) ? nkt + 1 : 0);
        pw_fence_proxy_async();  // the slot is refilled by TMA later
    };

    // coefficients of each level pair of the chunk, prepared once per CTA in
    // shared memory (keeps them out of the register file during the march):
    // per pair t: Gm, G0, GP0, GPp, R0, RP0 as float4 (hi pair, lo pair)
    float4 *ctab = reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(bars) + 64);
    for (int t = tid; t < nkt; t += nt) {
        const int N = g.cs_n;
        const int kq = min(k0 + 2 * t, g.nz - 1);  // pairs past the top read valid entries
        const D2 c6[6] = {cs_pair(cs, N, 0, kq - 1), cs_pair(cs, N, 0, kq), cs_pair(cs, N, 1, kq),
                          cs_pair(cs, N, 1, kq + 1), cs_pair(cs, N, 2, kq), cs_pair(cs, N, 3, kq)};
        for (int a = 0; a < 6; a++)
            ctab[t * 6 + a] = make_float4(lx(c6[a].h), ly(c6[a].h), lx(c6[a].l), ly(c6[a].l));
    }
    if (tid == 0) {
        const float *tc = cs + 8 * g.cs_n;
        ctab[nkt * 6] = make_float4(tc[0], tc[0], tc[1], tc[1]);
        ctab[nkt * 6 + 1] = make_float4(tc[2], tc[2], tc[3], tc[3]);
    }
    auto coef = [&](int a) {
        const float4 c = ctab[tk * 6 + a];
        return D2{pk(c.x, c.y), pk(c.z, c.w)};
    };
    auto tcoef = [&](int a) {
        const float4 c = ctab[nkt * 6 + a];
        return D2{pk(c.x, c.y), pk(c.z, c.w)};
    };
    const bool active = (j < g.ny) && (kbase < g.nz);

    // planes i0-1 and i0
    {
        const bool ok = wait(0) && wait(1);  // nplanes >= 3 always
        if (ok) {
            convert(0);
            convert(1);
        }
        if (!__syncthreads_and(ok)) {
            give_up(0);
            return;
        }
    }
    // x face sums of column i0-1|i0, carried along the march
    D2 Fx_m, Gx_m, Hx_m;
    {
        const double *Pm = planes, *Pc = planes + 3 * fs;  // planes 0 and 1 (slots 0, 1)
        const int rC = (tj + 1) * g.kb, rN = (tj + 2) * g.kb;
        const D2 uM0 = ld2<0>(Pm + rC, kk), uC0 = ld2<0>(Pc + rC, kk);
        Fx_m = df_add(uM0, uC0);
        Gx_m = df_add(uM0, ld2<0>(Pm + rN, kk));
        Hx_m = df_add(uM0, ld2<1>(Pm + rC, kk));
    }
    for (int i = i0; i < i_end; i++) {
        const int q = i - i0 + 1;
        bool ok = wait(q + 1);
        if (ok) convert(q + 1);
        if (!__syncthreads_and(ok)) {
            give_up(q + 1);
            return;
        }
        if (tid == 0 && q >= 2 && q - 2 + NS < nplanes) {
            issue(q - 2 + NS);
            issued = q - 1 + NS;
        }
        if (!active) continue;

        const double *Pm = planes + (size_t)((q - 1) % NS) * 3 * fs;
        const double *Pc = planes + (size_t)(q % NS) * 3 * fs;
        const double *Pp = planes + (size_t)((q + 1) % NS) * 3 * fs;
        const int rS = tj * g.kb, rC = (tj + 1) * g.kb, rN = (tj + 2) * g.kb;
        const double *uM = Pm + rC, *uC = Pc + rC, *uP = Pp + rC;
        const double *vMr = Pm + fs + rC, *vCr = Pc + fs + rC, *vPr = Pp + fs + rC;
        const double *wMr = Pm + 2 * fs + rC, *wCr = Pc + 2 * fs + rC, *wPr = Pp + 2 * fs + rC;

        // ---------------- su ----------------
        const D2 uM0 = ld2<0>(uM, kk), uC0 = ld2<0>(uC, kk), uP0 = ld2<0>(uP, kk);
        const D2 Fx_p = df_add(uC0, uP0);
        D2 X = df_mul(df_sub(df_mul(uM0, Fx_m), df_mul(uP0, Fx_p)), tcoef(0));
        const D2 uS0 = ld2<0>(Pc + rS, kk), uN0 = ld2<0>(Pc + rN, kk);
        const D2 vS0 = ld2<0>(Pc + fs + rS, kk), vSP0 = ld2<0>(Pp + fs + rS, kk);
        const D2 vC0 = ld2<0>(vCr, kk), vP0 = ld2<0>(vPr, kk);
        D2 Y = df_mul(df_sub(df_mul(uS0, df_add(vS0, vSP0)), df_mul(uN0, df_add(vC0, vP0))), tcoef(1));
        const D2 wCm = ld2<-1>(wCr, kk), wPm = ld2<-1>(wPr, kk);
        const D2 wC0 = ld2<0>(wCr, kk), wP0 = ld2<0>(wPr, kk);
        const D2 uCm = ld2<-1>(uC, kk), uCp = ld2<1>(uC, kk);
        D2 Z = df_mul(df_sub(df_mul(uCm, df_mul(df_add(wCm, wPm), coef(0))),
                             df_mul(uCp, df_mul(df_add(wC0, wP0), coef(1)))), coef(4));
        const D2 ru = df_add(df_add(X, Y), Z);

        // ---------------- sv ----------------
        const D2 vM0 = ld2<0>(vMr, kk), uNM0 = ld2<0>(Pm + rN, kk);
        const D2 Gx_p = df_add(uC0, uN0);
        X = df_mul(df_sub(df_mul(vM0, Gx_m), df_mul(vP0, Gx_p)), tcoef(0));
        const D2 vN0 = ld2<0>(Pc + fs + rN, kk);
        Y = df_mul(df_sub(df_mul(vS0, df_add(vS0, vC0)), df_mul(vN0, df_add(vC0, vN0))), tcoef(1));
        const D2 wNm = ld2<-1>(Pc + 2 * fs + rN, kk), wN0 = ld2<0>(Pc + 2 * fs + rN, kk);
        const D2 vCm = ld2<-1>(vCr, kk), vCp = ld2<1>(vCr, kk);
        Z = df_mul(df_sub(df_mul(vCm, df_mul(df_add(wCm, wNm), coef(0))),
                          df_mul(vCp, df_mul(df_add(wC0, wN0), coef(1)))), coef(4));
        const D2 rv = df_add(df_add(X, Y), Z);

        // ---------------- sw ----------------
        const D2 wM0 = ld2<0>(wMr, kk), uMp = ld2<1>(uM, kk);
        const D2 Hx_p = df_add(uC0, uCp);
        X = df_mul(df_sub(df_mul(wM0, Hx_m), df_mul(wP0, Hx_p)), tcoef(0));
        const D2 wS0 = ld2<0>(Pc + 2 * fs + rS, kk), vSp = ld2<1>(Pc + fs + rS, kk);
        Y = df_mul(df_sub(df_mul(wS0, df_add(vS0, vSp)), df_mul(wN0, df_add(vC0, vCp))), tcoef(1));
        const D2 wCp = ld2<1>(wCr, kk);
        Z = df_mul(df_sub(df_mul(wCm, df_mul(df_add(wCm, wC0), coef(2))),
                          df_mul(wCp, df_mul(df_add(wC0, wCp), coef(3)))), coef(5));
        const D2 rw = df_add(df_add(X, Y), Z);

        Fx_m = Fx_p;
        Gx_m = Gx_p;
        Hx_m = Hx_p;

        // ---------------- outputs ----------------
        const long long off = (long long)(i + 2) * g.si + (long long)(j + 2) * g.sj + kbase;
        double a0 = join(lx(ru.h), lx(ru.l)), a1 = join(ly(ru.h), ly(ru.l));
        double b0 = join(lx(rv.h), lx(rv.l)), b1 = join(ly(rv.h), ly(rv.l));
        double c0 = join(lx(rw.h), lx(rw.l)), c1 = join(ly(rw.h), ly(rw.l));
        if (kbase >= g.nz - 1) c0 = 0.0;
        if (kbase + 1 >= g.nz - 1) c1 = 0.0;
        if constexpr (STEP) {
            // x exactly from memory (the staged planes now hold (hi, lo) pairs);
            // the lid level of w is not a degree of freedom and stays 0
            const bool two = kbase + 1 < g.nz;
            double xu0 = xu[off], xv0 = xv[off], xw0 = xw[off];
            double xu1 = two ? xu[off + 1] : 0.0, xv1 = two ? xv[off + 1] : 0.0, xw1 = two ? xw[off + 1] : 0.0;
            if (kbase >= g.nz - 1) xw0 = 0.0;
            if (kbase + 1 >= g.nz - 1) xw1 = 0.0;
            const double ru2[2] = {fma(dt, a0, xu0), fma(dt, a1, xu1)};
            const double rv2[2] = {fma(dt, b0, xv0), fma(dt, b1, xv1)};
            const double rw2[2] = {fma(dt, c0, xw0), fma(dt, c1, xw1)};
            const int nvalid = g.nz - kbase;
            pw_store_images<double, 2>(su, i, j, kbase, ru2, nvalid, g.nx, g.ny, g.si, g.sj);
            pw_store_images<double, 2>(sv, i, j, kbase, rv2, nvalid, g.nx, g.ny, g.si, g.sj);
            pw_store_images<double, 2>(sw, i, j, kbase, rw2, nvalid, g.nx, g.ny, g.si, g.sj);
        } else if (kbase + 1 < g.nz) {
            double2 *pu = reinterpret_cast<double2 *>(su + off);
            double2 *pv = reinterpret_cast<double2 *>(sv + off);
            double2 *pw = reinterpret_cast<double2 *>(sw + off);
            if (BETA) {
                const double2 ou = *pu, ov = *pv, ow = *pw;
                a0 += ou.x; a1 += ou.y; b0 += ov.x; b1 += ov.y; c0 += ow.x; c1 += ow.y;
            }
            *pu = make_double2(a0, a1);
            *pv = make_double2(b0, b1);
            *pw = make_double2(c0, c1);
        } else {
            su[off] = BETA ? su[off] + a0 : a0;
            sv[off] = BETA ? sv[off] + b0 : b0;
            sw[off] = BETA ? sw[off] + c0 : c0;
        }
    }
    // every thread reaches this point (inactive ones only skip the arithmetic)
    if (__syncthreads_or(bad) && tid == 0) atomicOr(status + PW_STATUS_RANGE_WORD, 1);
}

static pw_status pw_launch_split(const pw_mesh *m, const void *u, const void *v, const void *w,
                                 void *su, void *sv, void *sw, int beta, cudaStream_t st,
                                 int tile_j, int tile_i, bool step, double dt) {
    constexpr int NS = 5;
    // compiled for 4 or 8 rows of columns per CTA (the nearest of the two is
    // used), with 64- or 32-level chunks: 128 threads per CTA either way
    tile_j = tile_j <= 5 ? 4 : 8;
    PwSplitGeom g;
    g.nx = m->nx;
    g.ny = m->ny;
    g.nz = m->nz;
    const int kc_one = (m->nz + 1) / 2 * 2, kc_max = tile_j == 4 ? 64 : 32;
    g.kc = kc_one <= kc_max ? kc_one : kc_max;
    g.kb = g.kc + 4;
    tile_i = pw_fit_tile_i(m, tile_i, (long)((m->ny + tile_j - 1) / tile_j) * ((m->nz + g.kc - 1) / g.kc));
    g.tj = tile_j;
    g.ti = tile_i;
    g.rows = 3 * (tile_j + 2);
    g.cpr = g.kb / 2;
    g.inv_cpr = 1.0f / (float)g.cpr;
    const int plane_elems = (tile_j + 2) * g.kb;
    g.field_stride = (plane_elems + 15) / 16 * 16;  // 128-byte aligned planes
    g.cs_n = m->nz + 4;
    g.si = m->si;
    g.sj = m->sj;
    const int threads = (g.kc / 2) * tile_j;
    if (threads > 256)
        return pw_fail(PW_ERR_SHAPE, "split kernel: tile_j=%d needs %d threads (max 256)", tile_j, threads);
    (void)NS;
    static_assert(NS * sizeof(uint64_t) <= 64, "barrier slot");
    const size_t smem = (size_t)NS * 3 * g.field_stride * 8 + 64 +
                        ((size_t)(g.kc / 2) * 6 + 2) * sizeof(float4);
    if (smem > 226 * 1024) return pw_fail(PW_ERR_SHAPE, "split kernel needs %zu bytes of shared memory", smem);
    CUtensorMap maps[3];
    const void *f[3] = {u, v, w};
    for (int q = 0; q < 3; q++) {
        pw_status s = pw_make_field_map(&maps[q], f[q], PW_F64, m->nx, m->ny, m->nzp, pw_kdim(m->nz, q), g.kb,
                                        tile_j + 2);
        if (s != PW_OK) return s;
    }
    auto kern = step ? (tile_j == 4 ? pw_advect_split_kernel<NS, 4, false, true>
                                    : pw_advect_split_kernel<NS, 8, false, true>)
                     : tile_j == 4 ? (beta ? pw_advect_split_kernel<NS, 4, true> : pw_advect_split_kernel<NS, 4, false>)
                                   : (beta ? pw_advect_split_kernel<NS, 8, true> : pw_advect_split_kernel<NS, 8, false>);
    PW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((unsigned)((m->nz + g.kc - 1) / g.kc), (unsigned)((m->ny + tile_j - 1) / tile_j),
              (unsigned)((m->nx + tile_i - 1) / tile_i));
    if (grid.y > 65535 || grid.z > 65535) return pw_fail(PW_ERR_SHAPE, "grid too large; raise tile_j or tile_i");
    kern<<<grid, threads, smem, st>>>(maps[0], maps[1], maps[2], (double *)su, (double *)sv, (double *)sw,
                                      m->coefsplit, g, m->status, (const double *)u, (const double *)v,
                                      (const double *)w, dt);
    PW_CUDA(cudaGetLastError());
    return PW_OK;
}

pw_status pw_launch_advect_split(const pw_mesh *m, const void *u, const void *v, const void *w,
                                 void *su, void *sv, void *sw, int beta, cudaStream_t st,
                                 int tile_j, int tile_i) {
    return pw_launch_split(m, u, v, w, su, sv, sw, beta, st, tile_j, tile_i, false, 0.0);
}

pw_status pw_launch_step_split(const pw_mesh *m, const void *u, const void *v, const void *w, void *un,
                               void *vn, void *wn, double dt, cudaStream_t st, int tile_j, int tile_i) {
    return pw_launch_split(m, u, v, w, un, vn, wn, 0, st, tile_j, tile_i, true, dt);
}
