// pw_scalars_split.cu -- PW advection of FP64 cell-centred scalars in
// double-float arithmetic on the FP32 pipe (the FP64 "split" path of
// pw_advect_split.cu applied to the scalar form of pw_scalars.cu).
//
// Native FP64 caps the scalar stencil near 50 G scalar-points/s on B300 (its
// FP64 units run ~1.7 operations per clock per SM).  Here the staged doubles are
// split into (hi, lo) float pairs by integer bit operations, the stencil runs in
// packed f32x2 double-float arithmetic over two levels, and each output is
// rebuilt with one FP64 add.
//
// Per step the wind-dependent factors are formed once and shared by the CTA's
// scalars:  HU_M = hx u(i-1), HU_C = hx u(i), HV_S = hy v(j-1), HV_C = hy v(j),
// A = 2 r(k) g(k-1) w(k-1), B = 2 r(k) g(k) w(k)   (hz1 = 2 g(k-1) r(k),
// hz2 = 2 g(k) r(k), g = 0.25 rho_w, r = 1/(rho_n dz)), so that
//   s = HU_M phi(i-1) - HU_C phi(i+1) + HV_S phi(j-1) - HV_C phi(j+1)
//     + A phi(k-1) - B phi(k+1).
// Levels at or above nz and the lid arrive from TMA as zeros (the tensor maps
// carry the logical k extent), as does the ground level k = -1.
//
// Layout (that of the wind kernel): a CTA owns TJ rows x a KC-level chunk and
// marches along x; thread (t, r) computes row r at levels k0 + t and
// k0 + t + KC/2, whose neighbours below and above are the level pairs of
// threads t - 1 and t + 1, so every operand is one aligned 16-byte shared load.
// TMA brings the raw (j,k) plane of u, v, w and the group's scalars into the
// raw slot; after a barrier the threads convert it out of place into a ring of
// two converted planes (16-byte chunk q of a row: (hi, hi, lo, lo) of levels
// (k0 + q - 1, k0 + q - 1 + KC/2)); after a second barrier the raw slot takes
// the next plane and the threads compute column i from converted planes i and
// i+1, with u and the scalars of column i-1 carried in registers.  The 8 x 32
// and 4 x 64 tiles are compiled with their geometry as constants; a generic
// instantiation (KC = 0) serves shorter columns.
#include <algorithm>

#include "pw_df.cuh"
#include "pw_internal.h"
#include "pw_march.cuh"  // pw_store_images

#define PW_SSPLIT_CONV 2  // converted planes (i, i+1)
#define PW_SSPLIT_GMAX 6  // scalars per CTA at most

struct PwScalarSplitSet {
    CUtensorMap phi[PW_MAX_SCALARS];
    double *out[PW_MAX_SCALARS];
    const double *in[PW_MAX_SCALARS];  // the scalars themselves (read exactly by the fused step)
};

struct PwScalarSplitGeom {
    int nx, ny, nz, kc, half, ti;
    int nkc, group, n;
    int rfs;           // doubles between the fields of the raw slot (128-byte aligned)
    int cs_n;          // levels in the coefficient table (nz + 4, level -2 first)
    long long si, sj;
};

// one level pair (a, b) of a converted row as hi and lo pairs
__device__ __forceinline__ D2 pw_ss_ldc(const float4 *row, int q) {
    const float4 c = row[q];
    return D2{pk(c.x, c.y), pk(c.z, c.w)};
}

// STEP: write phi + dt s (phi read exactly from set.in; the staged planes hold
// hi/lo pairs) at the column and at its periodic halo images
template <int TJ, int KC, bool BETA, int GMAX, bool STEP = false>
__global__ void __launch_bounds__(128, 4)
pw_scalar_split_kernel(const __grid_constant__ CUtensorMap mu, const __grid_constant__ CUtensorMap mv,
                       const __grid_constant__ CUtensorMap mw, const __grid_constant__ PwScalarSplitSet set,
                       const float *__restrict__ cs, const PwScalarSplitGeom g, int *__restrict__ status,
                       double dt = 0.0) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if (pw_cta_failed(status)) return;
    constexpr bool CT = KC > 0;
    constexpr int RFS_CT = CT ? ((TJ + 2) * (KC + 4) + 15) / 16 * 16 : 0;
    const int half = CT ? KC / 2 : g.half;
    const int cw = half + 2, kb = 2 * half + 4;
    const int rfs = CT ? RFS_CT : g.rfs;
    const int cfs = (TJ + 2) * cw;
    const int nt = CT ? (KC / 2) * TJ : (int)blockDim.x;
    // k chunks, then scalar groups, are the fastest grid indices: the chunks
    // and groups of one tile run together and share the wind planes in L2
    const int kchunk = blockIdx.x % g.nkc, grp = blockIdx.x / g.nkc;
    const int s0 = grp * g.group;
    const int G = min(g.group, g.n - s0);
    const int NF = 3 + G;
    double *raw = reinterpret_cast<double *>(smem_raw);
    float4 *conv = reinterpret_cast<float4 *>(smem_raw + (size_t)(3 + g.group) * rfs * 8);
    uint64_t *bars = reinterpret_cast<uint64_t *>(conv + (size_t)PW_SSPLIT_CONV * (3 + g.group) * cfs);
    float4 *ctab = reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(bars) + 64);
    const int tid = threadIdx.x;
    const int tk = tid % half, tj = tid / half;
    const int j0 = blockIdx.y * TJ, i0 = blockIdx.z * g.ti, k0 = kchunk * 2 * half;
    const int i_end = min(i0 + g.ti, g.nx);
    const int nplanes = i_end - i0 + 2;  // planes i0-1 .. i_end
    const uint32_t plane_bytes = (uint32_t)NF * (uint32_t)(TJ + 2) * (uint32_t)kb * 8u;
    const int ka = k0 + tk, kz = ka + half;  // this thread's two levels
    const int j = j0 + tj;

    if (tid == 0) {
        pw_prefetch_map(&mu);
        pw_prefetch_map(&mv);
        pw_prefetch_map(&mw);
        for (int q = 0; q < G; q++) pw_prefetch_map(&set.phi[s0 + q]);
        pw_mbar_init(&bars[0], 1);
        pw_fence_barrier_init();
    }
    __syncthreads();
    auto issue = [&](int p) {  // plane p (column i0-1+p) into the raw slot
        pw_mbar_expect_tx(&bars[0], plane_bytes);
        const int c0 = k0 - 2, c1 = j0 + 1, c2 = i0 + 1 + p;
        pw_tma_load_3d(raw, &mu, c0, c1, c2, &bars[0]);
        pw_tma_load_3d(raw + rfs, &mv, c0, c1, c2, &bars[0]);
        pw_tma_load_3d(raw + 2 * rfs, &mw, c0, c1, c2, &bars[0]);
        for (int q = 0; q < G; q++) pw_tma_load_3d(raw + (size_t)(3 + q) * rfs, &set.phi[s0 + q], c0, c1, c2, &bars[0]);
    };
    int issued = 0;
    if (tid == 0) {
        issue(0);
        issued = 1;
    }
    auto give_up = [&](int from) {
        if (tid == 0) {
            for (int p = from; p < issued; p++)
                if (!pw_mbar_wait_bounded(&bars[0], (uint32_t)(p & 1), PW_DRAIN_CYCLES)) break;
            atomicExch(status, (int)PW_ERR_TIMEOUT);
        }
    };

    // conversion of the raw plane into converted slot p % PW_SSPLIT_CONV: chunk q
    // of a row takes levels k0+q-1 and k0+q-1+half, i.e. raw positions q+1 and
    // q+1+half; thread (tk, tj) converts chunk tk+1 of rows tj, tj+TJ, ...; the
    // two edge chunks of each row (q = 0 and q = cw-1) are shared out
    bool bad = false;  // a value this thread converted was outside the split range
    const int rows = NF * (TJ + 2);
    auto conv_one = [&](int R, int q, float4 *cd) {
        const int f = R / (TJ + 2), r = R - f * (TJ + 2);
        const double *rs = raw + (size_t)f * rfs + r * kb + q + 1;
        const uint2 a = *reinterpret_cast<const uint2 *>(rs);
        const uint2 b = *reinterpret_cast<const uint2 *>(rs + half);
        // the winds (fields 0..2) and the scalars have their own ranges
        const uint32_t ehi = f < 3 ? PW_SPLIT_WIND_EHI : PW_SPLIT_SCALAR_EHI;
        float ha, la, hb, lb;
        split_words(a.x, a.y, ha, la, ehi, bad);
        split_words(b.x, b.y, hb, lb, ehi, bad);
        cd[(size_t)f * cfs + r * cw + q] = make_float4(ha, hb, la, lb);
    };
    auto convert = [&](int p) {
        float4 *cd = conv + (size_t)(p % PW_SSPLIT_CONV) * (3 + g.group) * cfs;
        for (int R = tj; R < rows; R += TJ) conv_one(R, tk + 1, cd);
        for (int e = tid; e < 2 * rows; e += nt) conv_one(e >> 1, (e & 1) ? cw - 1 : 0, cd);
        pw_fence_proxy_async();  // these reads come before the TMA refill of the raw slot
    };

    // coefficients of this thread's level pair, prepared once per CTA in shared
    // memory, coefficient-major (a warp's level pairs read contiguous bytes):
    // c * half + t holds g(k-1), g(k), 2 r(k) of levels (k0+t, k0+t+half) as
    // (hi, hi, lo, lo); then hx, hy
    auto cval = [&](int arr, int K) {  // (hi, lo) of table arr at level K
        const int N = g.cs_n;
        K = min(max(K, -2), g.nz + 1);
        return make_float2(cs[(2 * arr) * N + K + 2], cs[(2 * arr + 1) * N + K + 2]);
    };
    for (int t = tid; t < half; t += nt) {
        const int a = k0 + t, b = a + half;
        const float2 ga = cval(0, a - 1), gb = cval(0, b - 1);
        const float2 ha = cval(0, a), hb = cval(0, b);
        const float2 ra = cval(2, a), rb = cval(2, b);
        ctab[t] = make_float4(ga.x, gb.x, ga.y, gb.y);
        ctab[half + t] = make_float4(ha.x, hb.x, ha.y, hb.y);
        ctab[2 * half + t] = make_float4(2.0f * ra.x, 2.0f * rb.x, 2.0f * ra.y, 2.0f * rb.y);  // doubling is exact
    }
    if (tid == 0) {
        const float *tc = cs + 8 * g.cs_n;
        ctab[3 * half] = make_float4(2.0f * tc[0], 2.0f * tc[0], 2.0f * tc[1], 2.0f * tc[1]);
        ctab[3 * half + 1] = make_float4(2.0f * tc[2], 2.0f * tc[2], 2.0f * tc[3], 2.0f * tc[3]);
    }
    auto coef = [&](int c) { return pw_ss_ldc(ctab, c * half + tk); };
    const bool active = j < g.ny;
    const bool oka = ka < g.nz, okz = kz < g.nz;

    // operands: this thread's chunk of converted plane p, field f, row offset o
    // (0: j-1, 1: j, 2: j+1), level shift sh (-1, 0, +1)
    const int tb = tj * cw + tk + 1;
    auto base = [&](int p) { return conv + (size_t)(p % PW_SSPLIT_CONV) * (3 + g.group) * cfs + tb; };
    auto L = [&](const float4 *B, int f, int o, int sh) { return pw_ss_ldc(B, f * cfs + o * cw + sh); };

    D2 uM, pM[GMAX];  // u and the scalars of column i-1 (this thread's pair)
    for (int p = 0; p < nplanes; p++) {
        const bool ok = pw_mbar_wait_bounded(&bars[0], (uint32_t)(p & 1));
        // every thread is past step p-1 (which read converted plane p-2): its
        // slot takes plane p
        if (!__syncthreads_and(ok)) {
            give_up(p);
            return;
        }
        convert(p);
        __syncthreads();
        // every thread has converted plane p: the raw slot takes plane p + 1
        if (tid == 0 && p + 1 < nplanes) {
            issue(p + 1);
            issued = p + 2;
        }
        if (p == 0) {
            const float4 *B0 = base(0);
            uM = L(B0, 0, 1, 0);
#pragma unroll
            for (int s = 0; s < GMAX; s++)
                if (s < G) pM[s] = L(B0, 3 + s, 1, 0);
        }
        if (p < 2) continue;
        const int i = i0 + p - 2;  // the column computed now, from planes p-1 (C) and p (P)
        const float4 *BC = base(p - 1), *BP = base(p);
        // wind factors shared by the scalars
        const D2 hx = pw_ss_ldc(ctab, 3 * half), hy = pw_ss_ldc(ctab, 3 * half + 1);
        const D2 uC = L(BC, 0, 1, 0);
        const D2 HUm = df_mul(uM, hx), HUc = df_mul(uC, hx);
        const D2 HVs = df_mul(L(BC, 1, 0, 0), hy), HVc = df_mul(L(BC, 1, 1, 0), hy);
        const D2 r2 = coef(2);
        const D2 A = df_mul(df_mul(L(BC, 2, 1, -1), coef(0)), r2);
        const D2 B = df_mul(df_mul(L(BC, 2, 1, 0), coef(1)), r2);
        const long long off = (long long)(i + 2) * g.si + (long long)(j + 2) * g.sj;
#pragma unroll
        for (int s = 0; s < GMAX; s++) {
            if (s < G) {
                const int f = 3 + s;
                const D2 pC = L(BC, f, 1, 0);
                const D2 X = df_sub(df_mul(HUm, pM[s]), df_mul(HUc, L(BP, f, 1, 0)));
                const D2 Y = df_sub(df_mul(HVs, L(BC, f, 0, 0)), df_mul(HVc, L(BC, f, 2, 0)));
                const D2 Z = df_sub(df_mul(A, L(BC, f, 1, -1)), df_mul(B, L(BC, f, 1, 1)));
                const D2 r = df_add(df_add(X, Y), Z);
                pM[s] = pC;
                if (!active) continue;
                const double a0 = join(lx(r.h), lx(r.l)), a1 = join(ly(r.h), ly(r.l));
                if constexpr (STEP) {
                    const double *px = set.in[s0 + s] + off;
                    if (oka) {
                        const double o1[1] = {fma(dt, a0, px[ka])};
                        pw_store_images<double, 1>(set.out[s0 + s], i, j, ka, o1, 1, g.nx, g.ny, g.si, g.sj);
                    }
                    if (okz) {
                        const double o1[1] = {fma(dt, a1, px[kz])};
                        pw_store_images<double, 1>(set.out[s0 + s], i, j, kz, o1, 1, g.nx, g.ny, g.si, g.sj);
                    }
                } else {
                    double *po = set.out[s0 + s] + off;
                    if (oka) po[ka] = BETA ? po[ka] + a0 : a0;
                    if (okz) po[kz] = BETA ? po[kz] + a1 : a1;
                }
            }
        }
        uM = uC;
    }
    // every thread reaches this point (inactive rows only skip the stores)
    if (__syncthreads_or(bad) && tid == 0) atomicOr(status + PW_STATUS_RANGE_WORD, 1);
    if (tid == 0) pw_mbar_inval(&bars[0]);
}

pw_status pw_launch_scalars_split(const pw_mesh *m, const void *u, const void *v, const void *w, int n,
                                  const void *const *phi, void *const *sphi, int beta, cudaStream_t st,
                                  int tile_j, int tile_i, int group, bool step, double dt) {
    // compiled for 4 or 8 rows of columns per CTA (the nearest of the two is
    // used), with 64- or 32-level chunks: 128 threads per CTA
    tile_j = tile_j <= 5 ? 4 : 8;
    PwScalarSplitGeom g;
    g.nx = m->nx;
    g.ny = m->ny;
    g.nz = m->nz;
    const int kc_one = (m->nz + 1) / 2 * 2, kc_max = tile_j == 4 ? 64 : 32;
    g.kc = kc_one <= kc_max ? kc_one : kc_max;
    g.half = g.kc / 2;
    const int kb = g.kc + 4, cw = g.half + 2;
    g.rfs = ((tile_j + 2) * kb + 15) / 16 * 16;  // 128-byte aligned TMA destinations
    g.cs_n = m->nz + 4;
    g.si = m->si;
    g.sj = m->sj;
    const int threads = g.half * tile_j;
    // per field: the raw slot and two converted planes
    const size_t field_bytes = (size_t)g.rfs * 8 + (size_t)PW_SSPLIT_CONV * (tile_j + 2) * cw * 16;
    const size_t fixed = 64 + ((size_t)g.half * 3 + 2) * sizeof(float4);
    if (group <= 0) {
        // the largest group whose CTA still lets 4 CTAs share an SM (228 KB of
        // shared memory, 1 KB of it reserved per CTA): the double-float arithmetic
        // needs the warps to hide its latency, so two groups of three scalars at 16
        // warps per SM beat one group of six at 8 although the wind is staged twice
        const long fit = (long)(226 * 1024 - fixed) / (long)field_bytes - 3;
        const long fit4 = (long)(56 * 1024 - fixed) / (long)field_bytes - 3;
        const long gmax = std::min((long)std::min(n, PW_SSPLIT_GMAX), fit);
        group = (int)std::max(1L, fit4 >= 1 ? std::min(gmax, fit4) : gmax);
        const int ngroups = (n + group - 1) / group;
        group = (n + ngroups - 1) / ngroups;
    }
    group = std::min(std::min(group, n), PW_SSPLIT_GMAX);
    g.group = group;
    g.n = n;
    g.nkc = (m->nz + g.kc - 1) / g.kc;
    const size_t smem = field_bytes * (size_t)(3 + group) + fixed;
    if (smem > 226 * 1024)
        return pw_fail(PW_ERR_SHAPE, "scalar split kernel needs %zu bytes of shared memory", smem);
    CUtensorMap maps[3];
    const void *f[3] = {u, v, w};
    for (int q = 0; q < 3; q++) {
        pw_status s = pw_make_field_map(&maps[q], f[q], PW_F64, m->nx, m->ny, m->nzp, pw_kdim(m->nz, q), kb,
                                        tile_j + 2);
        if (s != PW_OK) return s;
    }
    PwScalarSplitSet set;
    memset(&set, 0, sizeof(set));
    for (int q = 0; q < n; q++) {
        pw_status s = pw_make_field_map(&set.phi[q], phi[q], PW_F64, m->nx, m->ny, m->nzp, m->nz, kb, tile_j + 2);
        if (s != PW_OK) return s;
        set.out[q] = (double *)sphi[q];
        set.in[q] = (const double *)phi[q];
    }
    constexpr int GM = PW_SSPLIT_GMAX;
    const bool full = g.kc == kc_max;
    using KernT = decltype(&pw_scalar_split_kernel<8, 32, false, GM>);
    KernT kern;
#define PW_SS_PICK(TJ, KC)                                                               \
    (step ? pw_scalar_split_kernel<TJ, KC, false, GM, true>                              \
          : beta ? pw_scalar_split_kernel<TJ, KC, true, GM> : pw_scalar_split_kernel<TJ, KC, false, GM>)
    if (tile_j == 8) kern = full ? PW_SS_PICK(8, 32) : PW_SS_PICK(8, 0);
    else kern = full ? PW_SS_PICK(4, 64) : PW_SS_PICK(4, 0);
#undef PW_SS_PICK
    PW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long ngroups = (n + group - 1) / group;
    // the fill rule (the wave rule of pw_pick_tile_i measured no faster on
    // these many-wave grids)
    tile_i = pw_fit_tile_i(m, tile_i, (long)((m->ny + tile_j - 1) / tile_j) * g.nkc);
    g.ti = tile_i;
    dim3 grid((unsigned)(g.nkc * ngroups), (unsigned)((m->ny + tile_j - 1) / tile_j),
              (unsigned)((m->nx + tile_i - 1) / tile_i));
    if (grid.y > 65535 || grid.z > 65535) return pw_fail(PW_ERR_SHAPE, "grid too large; raise tile_j or tile_i");
    kern<<<grid, threads, smem, st>>>(maps[0], maps[1], maps[2], set, m->coefsplit, g, m->status, dt);
    PW_CUDA(cudaGetLastError());
    return PW_OK;
}
