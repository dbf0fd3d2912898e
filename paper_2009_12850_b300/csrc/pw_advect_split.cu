// pw_advect_split.cu -- FP64 PW stencil in double-float arithmetic (FP64 in,
// FP64 out, error within a few units of 2^-46 of the per-point condition sum).
//
// Why: B300's FP64 units run at ~1.6 operations / clock / SM, so native FP64
// caps this ~42-FLOP-per-point stencil near 11 Gpoints/s (8% of the HBM
// roofline).  Here every double is split exactly-enough into two floats and the
// stencil runs on the FP32 pipe (packed .f32x2 instructions over two levels of
// a column), with FP64 used only for one add per output.
//
// Layout of the work: an x-march.  A CTA owns TJ rows of columns and a k chunk
// of KC levels (8 rows x 32 levels by default, or 4 x 64); the k chunk is the
// fastest grid index, so the chunks of a column run together and the k-halo
// levels they share come from L2.  Thread (t, r) computes row r at the two
// levels k0 + t and k0 + t + KC/2: with that pairing the level pairs one below
// and one above it are the pairs of its neighbours t - 1 and t + 1, so every
// operand of the stencil is one aligned 16-byte load from shared memory.
//
// Pipeline per x step: TMA brings the (j,k) plane of u, v, w (doubles, rows
// j0-1 .. j0+TJ, levels k0-2 .. k0+KC+1; levels >= nz and the w lid arrive as
// zeros because the tensor maps carry the logical k extent) into the raw slot;
// all threads convert it, with integer bit operations, into a ring of four
// converted planes whose 16-byte chunk q of a row holds (hi, hi, lo, lo) of
// levels (k0 + q - 1, k0 + q - 1 + KC/2); after the step's one barrier the raw
// slot takes the next plane (its copy runs during the arithmetic) and the
// threads compute column i from converted planes i-1, i, i+1 (the fourth is
// the one the next step writes, so no barrier is needed before converting).
// One raw slot and four converted planes (44 KB for the 8 x 32 tile) let five
// CTAs share an SM.
//
// The algebra: s = tcx X + tcy Y + Z with X, Y differences of products of a
// field value and a face sum, and Z = phi(k-1) (A(k-1) c1) - phi(k+1) (A(k) c2)
// with the vertical coefficients c1, c2 (tzc1, tzc2 or tzd1, tzd2) applied to
// the face sums A; when tcx == tcy (a square horizontal grid) s = tcx (X + Y) + Z.
#include <algorithm>

#include "pw_df.cuh"
#include "pw_internal.h"
#include "pw_march.cuh"  // pw_store_images

struct PwSplitGeom {
    int nx, ny, nz;
    int kc, half;      // levels per CTA chunk (even), kc / 2
    int kb;            // raw row length in doubles: kc + 4 (levels k0-2 .. k0+kc+1)
    int cw;            // converted chunks per row: half + 2
    int ti;            // columns marched per CTA
    int rfs;           // doubles between the u, v, w planes of a raw slot (128-byte aligned)
    int cfs;           // 16-byte chunks between the u, v, w planes of a converted slot
    long long si, sj;
    double tcx, tcy;
};

#define PW_SPLIT_RAW 1   // raw TMA slots
#define PW_SPLIT_CONV 4  // converted planes (i-1, i, i+1 and the one being written)

// one level pair (a, b) of a converted row as hi and lo pairs
__device__ __forceinline__ D2 pw_ldc(const float4 *row, int q) {
    const float4 c = row[q];
    return D2{pk(c.x, c.y), pk(c.z, c.w)};
}

// STEP: write x + dt S(x) (x read exactly from xu, xv, xw) to su, sv, sw and to
// their periodic halo images, the forward Euler step fused into the stencil
template <int TJ, int KC, bool BETA, bool STEP = false, bool ISO = false>
__global__ void __launch_bounds__(128, 5)
pw_advect_split_kernel(const __grid_constant__ CUtensorMap mu, const __grid_constant__ CUtensorMap mv,
                       const __grid_constant__ CUtensorMap mw, double *__restrict__ su,
                       double *__restrict__ sv, double *__restrict__ sw,
                       const double *__restrict__ cz, const PwSplitGeom g,
                       int *__restrict__ status, const double *__restrict__ xu = nullptr,
                       const double *__restrict__ xv = nullptr, const double *__restrict__ xw = nullptr,
                       double dt = 0.0) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int ROWS = 3 * (TJ + 2);
    // geometry: compile-time constants for the 8 x 32 and 4 x 64 tiles (every
    // shared-memory operand is then a base register plus an immediate offset),
    // from g for the short columns
    constexpr bool CT = KC > 0;
    constexpr int RFS_CT = CT ? ((TJ + 2) * (KC + 4) + 15) / 16 * 16 : 0;
    const int half = CT ? KC / 2 : g.half;
    const int cw = half + 2, kb = 2 * half + 4;
    const int rfs = CT ? RFS_CT : g.rfs;
    const int cfs = (TJ + 2) * cw;
    const int nt = CT ? (KC / 2) * TJ : (int)blockDim.x;
    double *raw = reinterpret_cast<double *>(smem_raw);
    float4 *conv = reinterpret_cast<float4 *>(smem_raw + (size_t)PW_SPLIT_RAW * 3 * rfs * 8);
    uint64_t *bars = reinterpret_cast<uint64_t *>(conv + (size_t)PW_SPLIT_CONV * 3 * cfs);
    float4 *ctab = reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(bars) + 64);
    const int tid = threadIdx.x;
    const int tk = tid % half, tj = tid / half;
    // k chunks are the fastest grid index: the chunks of a column run together,
    // so the k-halo levels they share are fetched from DRAM once (L2 hits)
    const int j0 = blockIdx.y * TJ, i0 = blockIdx.z * g.ti, k0 = blockIdx.x * 2 * half;
    const int i_end = min(i0 + g.ti, g.nx);
    const int nplanes = i_end - i0 + 2;
    const uint32_t plane_bytes = 3u * (uint32_t)(TJ + 2) * (uint32_t)kb * 8u;
    const int ka = k0 + tk, kz = ka + half;  // this thread's two levels
    const int j = j0 + tj;

    if (pw_cta_failed(status)) return;
    if (tid == 0) {
        pw_prefetch_map(&mu);
        pw_prefetch_map(&mv);
        pw_prefetch_map(&mw);
        for (int s = 0; s < PW_SPLIT_RAW; s++) pw_mbar_init(&bars[s], 1);
        pw_fence_barrier_init();
    }
    __syncthreads();
    auto issue = [&](int p) {
        const int s = p % PW_SPLIT_RAW;
        double *dst = raw + (size_t)s * 3 * rfs;
        pw_mbar_expect_tx(&bars[s], plane_bytes);
        const int c0 = k0 - 2, c1 = j0 + 1, c2 = i0 + 1 + p;
        pw_tma_load_3d(dst, &mu, c0, c1, c2, &bars[s]);
        pw_tma_load_3d(dst + rfs, &mv, c0, c1, c2, &bars[s]);
        pw_tma_load_3d(dst + 2 * rfs, &mw, c0, c1, c2, &bars[s]);
    };
    int issued = 0;
    if (tid == 0) {
        for (int p = 0; p < min(PW_SPLIT_RAW, nplanes); p++) issue(p);
        issued = min(PW_SPLIT_RAW, nplanes);
    }
    auto give_up = [&](int from) {
        if (tid == 0) {
            for (int p = from; p < issued; p++)
                if (!pw_mbar_wait_bounded(&bars[p % PW_SPLIT_RAW], (uint32_t)((p / PW_SPLIT_RAW) & 1),
                                          PW_DRAIN_CYCLES))
                    break;
            atomicExch(status, (int)PW_ERR_TIMEOUT);
        }
    };

    // conversion of raw plane p into converted slot p % PW_SPLIT_CONV: chunk q
    // of a row takes levels k0+q-1 and k0+q-1+half, i.e. raw positions q+1 and
    // q+1+half.  Thread (tk, tj) converts chunk tk+1 of rows tj, tj+TJ, ...; the
    // two edge chunks of each row (q = 0 and q = cw-1) are shared out.
    bool bad = false;  // a value this thread converted was outside the split range
    constexpr int MR = (ROWS + TJ - 1) / TJ;  // rows of main chunks per thread
    auto src_of = [&](int R, int q) {
        const int f = (R >= TJ + 2) + (R >= 2 * (TJ + 2));
        return f * rfs + (R - f * (TJ + 2)) * kb + q + 1;
    };
    int soff[MR], doff[MR];
#pragma unroll
    for (int m = 0; m < MR; m++) {
        const int R = min(tj + m * TJ, ROWS - 1);
        soff[m] = src_of(R, tk + 1);
        doff[m] = R * cw + tk + 1;
    }
    // this thread's edge chunk (fixed tiles): 8 x 32: warp 3 (rows 6, 7: three
    // main rows each) takes edges 0-31, warps 0-2 share the other 28;
    // 4 x 64: warps 2, 3 (four main rows) take the 36 edges
    int edge = -1;
    if constexpr (CT) {
        const int warp = tid >> 5, lane = tid & 31;
        if (TJ == 8) edge = warp == 3 ? lane : (lane * 3 + warp < 2 * ROWS - 32 ? 32 + lane * 3 + warp : -1);
        else edge = warp >= 2 && (warp - 2) * 32 + lane < 2 * ROWS ? (warp - 2) * 32 + lane : -1;
    }
    const int esrc = edge >= 0 ? src_of(edge >> 1, (edge & 1) ? cw - 1 : 0) : 0;
    auto conv_one = [&](const double *rs, float4 *cd, int so, int dof) {
        const uint2 a = *reinterpret_cast<const uint2 *>(rs + so);
        const uint2 b = *reinterpret_cast<const uint2 *>(rs + so + half);
        float ha, la, hb, lb;
        split_words(a.x, a.y, ha, la, PW_SPLIT_WIND_EHI, bad);
        split_words(b.x, b.y, hb, lb, PW_SPLIT_WIND_EHI, bad);
        cd[dof] = make_float4(ha, hb, la, lb);
    };
    auto convert = [&](int p) {
        const double *rs = raw + (size_t)(p % PW_SPLIT_RAW) * 3 * rfs;
        float4 *cd = conv + (size_t)(p % PW_SPLIT_CONV) * 3 * cfs;
#pragma unroll
        for (int m = 0; m < MR; m++)
            if (m + 1 < MR || tj + m * TJ < ROWS) conv_one(rs, cd, soff[m], doff[m]);
        // the two edge chunks of each row (q = 0 and q = cw-1): for the fixed
        // tiles, handed first to the warps with fewer main rows (so that every
        // warp reaches the barrier with about the same work)
        if constexpr (CT) {
            if (edge >= 0) {
                const int R = edge >> 1, q = (edge & 1) ? cw - 1 : 0;
                conv_one(rs, cd, esrc, R * cw + q);
            }
        } else {
            for (int e = tid; e < 2 * ROWS; e += nt) {
                const int R = e >> 1, q = (e & 1) ? cw - 1 : 0;
                conv_one(rs, cd, src_of(R, q), R * cw + q);
            }
        }
        pw_fence_proxy_async();  // these reads come before the TMA refill of the slot
    };

    // coefficients of this thread's level pair, prepared once per CTA in shared
    // memory (keeps them out of the register file during the march): per
    // thread column tk: tzc1, tzc2, tzd1, tzd2 of levels (ka, kz) as float4
    // (hi pair, lo pair), split from the FP64 table; then tcx, tcy
    auto cpair = [](double c) {
        const float h = (float)c;
        return make_float2(h, (float)(c - (double)h));
    };
    for (int t = tid; t < half; t += nt) {
        const int a = k0 + t, b = a + half;
        for (int c = 0; c < 4; c++) {
            const float2 x = cpair(a < g.nz ? cz[c * g.nz + a] : 0.0);
            const float2 y = cpair(b < g.nz ? cz[c * g.nz + b] : 0.0);
            ctab[c * half + t] = make_float4(x.x, y.x, x.y, y.y);
        }
    }
    if (tid == 0) {
        const float2 x = cpair(g.tcx), y = cpair(g.tcy);
        ctab[half * 4] = make_float4(x.x, x.x, x.y, x.y);
        ctab[half * 4 + 1] = make_float4(y.x, y.x, y.y, y.y);
    }
    // coefficient a of level pair t at a * half + t: a warp's 16 level pairs
    // read 256 contiguous bytes (conflict-free)
    auto coef = [&](int a) { return pw_ldc(ctab, a * half + tk); };
    auto tcoef = [&](int a) { return pw_ldc(ctab, half * 4 + a); };
    const bool active = j < g.ny;
    const bool oka = ka < g.nz, okz = kz < g.nz;

    // operands: this thread's chunk of plane p, field f, row offset o (0: j-1,
    // 1: j, 2: j+1), level shift sh (-1, 0, +1)
    const int tb = tj * cw + tk + 1;
    auto base = [&](int p) { return conv + (size_t)(p % PW_SPLIT_CONV) * 3 * cfs + tb; };
    auto L = [&](const float4 *B, int f, int o, int sh) { return pw_ldc(B, f * cfs + o * cw + sh); };

    // tcx X + tcy Y + Z; with tcx == tcy (a square horizontal grid) one product
    // (the table is read after the first barrier of the march)
    auto horiz = [&](D2 X, D2 Y, D2 Z) {
        if constexpr (ISO) return df_add(df_mul(df_add(X, Y), tcoef(0)), Z);
        else return df_add(df_add(df_mul(X, tcoef(0)), df_mul(Y, tcoef(1))), Z);
    };
    D2 Fx_m, Gx_m, Hx_m;  // x face sums of column i-1|i, carried along the march
    for (int p = 0; p < nplanes; p++) {
        const bool ok = pw_mbar_wait_bounded(&bars[p % PW_SPLIT_RAW], (uint32_t)((p / PW_SPLIT_RAW) & 1));
        if (ok) convert(p);
        // one barrier per step: plane p is published and its raw slot free, and
        // every thread is past step p-1, so the converted plane the next step
        // overwrites (p-3) is no longer read
        if (!__syncthreads_and(ok)) {
            give_up(p);
            return;
        }
        // every thread has converted plane p: its raw slot takes plane p + 1
        if (tid == 0 && p + PW_SPLIT_RAW < nplanes) {
            issue(p + PW_SPLIT_RAW);
            issued = p + PW_SPLIT_RAW + 1;
        }
        if (p == 1) {
            const float4 *B0 = base(0), *B1 = base(1);
            const D2 uM0 = L(B0, 0, 1, 0);
            Fx_m = df_add(uM0, L(B1, 0, 1, 0));
            Gx_m = df_add(uM0, L(B0, 0, 2, 0));
            Hx_m = df_add(uM0, L(B0, 0, 1, 1));
        }
        if (p < 2) continue;
        const int i = i0 + p - 2;  // the column computed now, from planes p-2, p-1, p
        const float4 *BM = base(p - 2), *BC = base(p - 1), *BP = base(p);

        // ---------------- su ----------------
        const D2 uM0 = L(BM, 0, 1, 0), uC0 = L(BC, 0, 1, 0), uP0 = L(BP, 0, 1, 0);
        const D2 Fx_p = df_add(uC0, uP0);
        D2 X = df_sub(df_mul(uM0, Fx_m), df_mul(uP0, Fx_p));
        const D2 uS0 = L(BC, 0, 0, 0), uN0 = L(BC, 0, 2, 0);
        const D2 vS0 = L(BC, 1, 0, 0), vSP0 = L(BP, 1, 0, 0);
        const D2 vC0 = L(BC, 1, 1, 0), vP0 = L(BP, 1, 1, 0);
        D2 Y = df_sub(df_mul(uS0, df_add(vS0, vSP0)), df_mul(uN0, df_add(vC0, vP0)));
        const D2 wCm = L(BC, 2, 1, -1), wPm = L(BP, 2, 1, -1);
        const D2 wC0 = L(BC, 2, 1, 0), wP0 = L(BP, 2, 1, 0);
        const D2 uCm = L(BC, 0, 1, -1), uCp = L(BC, 0, 1, 1);
        D2 Z = df_sub(df_mul(uCm, df_mul(df_add(wCm, wPm), coef(0))), df_mul(uCp, df_mul(df_add(wC0, wP0), coef(1))));
        const D2 ru = horiz(X, Y, Z);

        // ---------------- sv ----------------
        const D2 vM0 = L(BM, 1, 1, 0);
        const D2 Gx_p = df_add(uC0, uN0);
        X = df_sub(df_mul(vM0, Gx_m), df_mul(vP0, Gx_p));
        const D2 vN0 = L(BC, 1, 2, 0);
        Y = df_sub(df_mul(vS0, df_add(vS0, vC0)), df_mul(vN0, df_add(vC0, vN0)));
        const D2 wNm = L(BC, 2, 2, -1), wN0 = L(BC, 2, 2, 0);
        const D2 vCm = L(BC, 1, 1, -1), vCp = L(BC, 1, 1, 1);
        Z = df_sub(df_mul(vCm, df_mul(df_add(wCm, wNm), coef(0))), df_mul(vCp, df_mul(df_add(wC0, wN0), coef(1))));
        const D2 rv = horiz(X, Y, Z);

        // ---------------- sw ----------------
        const D2 wM0 = L(BM, 2, 1, 0);
        const D2 Hx_p = df_add(uC0, uCp);
        X = df_sub(df_mul(wM0, Hx_m), df_mul(wP0, Hx_p));
        const D2 wS0 = L(BC, 2, 0, 0), vSp = L(BC, 1, 0, 1);
        Y = df_sub(df_mul(wS0, df_add(vS0, vSp)), df_mul(wN0, df_add(vC0, vCp)));
        const D2 wCp = L(BC, 2, 1, 1);
        Z = df_sub(df_mul(wCm, df_mul(df_add(wCm, wC0), coef(2))), df_mul(wCp, df_mul(df_add(wC0, wCp), coef(3))));
        const D2 rw = horiz(X, Y, Z);

        Fx_m = Fx_p;
        Gx_m = Gx_p;
        Hx_m = Hx_p;
        if (!active) continue;

        // ---------------- outputs: levels ka and kz ----------------
        const long long off = (long long)(i + 2) * g.si + (long long)(j + 2) * g.sj;
        double a0 = join(lx(ru.h), lx(ru.l)), a1 = join(ly(ru.h), ly(ru.l));
        double b0 = join(lx(rv.h), lx(rv.l)), b1 = join(ly(rv.h), ly(rv.l));
        double e0 = join(lx(rw.h), lx(rw.l)), e1 = join(ly(rw.h), ly(rw.l));
        if (ka >= g.nz - 1) e0 = 0.0;  // the lid face (and above)
        if (kz >= g.nz - 1) e1 = 0.0;
        if constexpr (STEP) {
            // x exactly from memory; the lid level of w stays 0
            if (oka) {
                const long long o = off + ka;
                const double xw0 = ka >= g.nz - 1 ? 0.0 : xw[o];
                const double r0[1] = {fma(dt, a0, xu[o])}, r1[1] = {fma(dt, b0, xv[o])},
                             r2[1] = {fma(dt, e0, xw0)};
                pw_store_images<double, 1>(su, i, j, ka, r0, 1, g.nx, g.ny, g.si, g.sj);
                pw_store_images<double, 1>(sv, i, j, ka, r1, 1, g.nx, g.ny, g.si, g.sj);
                pw_store_images<double, 1>(sw, i, j, ka, r2, 1, g.nx, g.ny, g.si, g.sj);
            }
            if (okz) {
                const long long o = off + kz;
                const double xw1 = kz >= g.nz - 1 ? 0.0 : xw[o];
                const double r0[1] = {fma(dt, a1, xu[o])}, r1[1] = {fma(dt, b1, xv[o])},
                             r2[1] = {fma(dt, e1, xw1)};
                pw_store_images<double, 1>(su, i, j, kz, r0, 1, g.nx, g.ny, g.si, g.sj);
                pw_store_images<double, 1>(sv, i, j, kz, r1, 1, g.nx, g.ny, g.si, g.sj);
                pw_store_images<double, 1>(sw, i, j, kz, r2, 1, g.nx, g.ny, g.si, g.sj);
            }
        } else {
            if (oka) {
                double *pu = su + off + ka, *pv = sv + off + ka, *pw = sw + off + ka;
                *pu = BETA ? *pu + a0 : a0;
                *pv = BETA ? *pv + b0 : b0;
                *pw = BETA ? *pw + e0 : e0;
            }
            if (okz) {
                double *pu = su + off + kz, *pv = sv + off + kz, *pw = sw + off + kz;
                *pu = BETA ? *pu + a1 : a1;
                *pv = BETA ? *pv + b1 : b1;
                *pw = BETA ? *pw + e1 : e1;
            }
        }
    }
    // every thread reaches this point (inactive rows only skip the stores)
    if (__syncthreads_or(bad) && tid == 0) atomicOr(status + PW_STATUS_RANGE_WORD, 1);
}

static pw_status pw_launch_split(const pw_mesh *m, const void *u, const void *v, const void *w,
                                 void *su, void *sv, void *sw, int beta, cudaStream_t st,
                                 int tile_j, int tile_i, bool step, double dt) {
    // compiled for 4 or 8 rows of columns per CTA (the nearest of the two is
    // used), with 64- or 32-level chunks: at most 128 threads per CTA
    tile_j = tile_j <= 5 ? 4 : 8;
    PwSplitGeom g;
    g.nx = m->nx;
    g.ny = m->ny;
    g.nz = m->nz;
    const int kc_one = (m->nz + 1) / 2 * 2, kc_max = tile_j == 4 ? 64 : 32;
    g.kc = kc_one <= kc_max ? kc_one : kc_max;
    g.half = g.kc / 2;
    g.kb = g.kc + 4;
    g.cw = g.half + 2;
    const long tiles = (long)((m->ny + tile_j - 1) / tile_j) * ((m->nz + g.kc - 1) / g.kc);
    g.rfs = ((tile_j + 2) * g.kb + 15) / 16 * 16;  // 128-byte aligned TMA destinations
    g.cfs = (tile_j + 2) * g.cw;
    g.si = m->si;
    g.sj = m->sj;
    g.tcx = m->tcx;
    g.tcy = m->tcy;
    const int threads = g.half * tile_j;
    if (threads > 128)
        return pw_fail(PW_ERR_SHAPE, "split kernel: tile_j=%d needs %d threads (max 128)", tile_j, threads);
    const size_t smem = (size_t)PW_SPLIT_RAW * 3 * g.rfs * 8 + (size_t)PW_SPLIT_CONV * 3 * g.cfs * 16 + 64 +
                        ((size_t)g.half * 4 + 2) * sizeof(float4);
    if (smem > 226 * 1024) return pw_fail(PW_ERR_SHAPE, "split kernel needs %zu bytes of shared memory", smem);
    CUtensorMap maps[3];
    const void *f[3] = {u, v, w};
    for (int q = 0; q < 3; q++) {
        pw_status s = pw_make_field_map(&maps[q], f[q], PW_F64, m->nx, m->ny, m->nzp, pw_kdim(m->nz, q), g.kb,
                                        tile_j + 2);
        if (s != PW_OK) return s;
    }
    // compile-time geometry for the full 8 x 32 and 4 x 64 tiles, the generic
    // instantiation (KC = 0) for shorter columns
    const bool full = g.kc == kc_max;
    using KernT = decltype(&pw_advect_split_kernel<8, 32, false, false>);
    KernT kern;
    const bool iso = m->tcx == m->tcy;
#define PW_SPLIT_PICK(TJ, KC)                                                                        \
    (step ? (iso ? pw_advect_split_kernel<TJ, KC, false, true, true> : pw_advect_split_kernel<TJ, KC, false, true>) \
     : beta ? (iso ? pw_advect_split_kernel<TJ, KC, true, false, true> : pw_advect_split_kernel<TJ, KC, true>)     \
            : (iso ? pw_advect_split_kernel<TJ, KC, false, false, true> : pw_advect_split_kernel<TJ, KC, false>))
    if (tile_j == 8) kern = full ? PW_SPLIT_PICK(8, 32) : PW_SPLIT_PICK(8, 0);
    else kern = full ? PW_SPLIT_PICK(4, 64) : PW_SPLIT_PICK(4, 0);
#undef PW_SPLIT_PICK
    PW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // a CTA marches ti columns from ti + 2 planes
    tile_i = pw_pick_tile_i(m, tile_i, tiles, pw_slots(m, kern, threads, smem), 2);
    g.ti = tile_i;
    dim3 grid((unsigned)((m->nz + g.kc - 1) / g.kc), (unsigned)((m->ny + tile_j - 1) / tile_j),
              (unsigned)((m->nx + tile_i - 1) / tile_i));
    if (grid.y > 65535 || grid.z > 65535) return pw_fail(PW_ERR_SHAPE, "grid too large; raise tile_j or tile_i");
    kern<<<grid, threads, smem, st>>>(maps[0], maps[1], maps[2], (double *)su, (double *)sv, (double *)sw,
                                      m->coef64 + 6 * m->nz, g, m->status, (const double *)u, (const double *)v,
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
