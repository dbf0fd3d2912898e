// pw_scalars_split.cu -- PW advection of FP64 cell-centred scalars in
// double-float arithmetic on the FP32 pipe (the FP64 "split" path of
// pw_advect_split.cu applied to the scalar form of pw_scalars.cu).
//
// Native FP64 caps the scalar stencil near 50 G scalar-points/s on B300 (its
// FP64 units run ~1.7 operations per clock per SM).  Here the staged doubles are
// split in place into (hi, lo) float pairs by integer bit operations, the
// stencil runs in packed f32x2 double-float arithmetic over two levels, and each
// output is rebuilt with one FP64 add.
//
// Per step the wind-dependent factors are formed once and shared by the CTA's
// scalars:  HU_M = hx u(i-1), HU_C = hx u(i), HV_S = hy v(j-1), HV_C = hy v(j),
// A = 2 r(k) g(k-1) w(k-1), B = 2 r(k) g(k) w(k)   (hz1 = 2 g(k-1) r(k),
// hz2 = 2 g(k) r(k), g = 0.25 rho_w, r = 1/(rho_n dz)), so that
//   s = HU_M phi(i-1) - HU_C phi(i+1) + HV_S phi(j-1) - HV_C phi(j+1)
//     + A phi(k-1) - B phi(k+1).
// Levels at or above nz and the lid arrive from TMA as zeros (the tensor maps
// carry the logical k extent), as does the ground level k = -1.
#include <algorithm>

#include "pw_df.cuh"
#include "pw_internal.h"
#include "pw_march.cuh"  // pw_store_images

#define PW_SSPLIT_NS 3    // planes i, i+1 and the one in flight
#define PW_SSPLIT_GMAX 6  // scalars per CTA at most

struct PwScalarSplitSet {
    CUtensorMap phi[PW_MAX_SCALARS];
    double *out[PW_MAX_SCALARS];
    const double *in[PW_MAX_SCALARS];  // the scalars themselves (read exactly by the fused step)
};

struct PwScalarSplitGeom {
    int nx, ny, nz, kc, kb, ti;
    int nkc, group, n;
    int field_stride;  // doubles between the fields of a slot
    int cs_n;          // levels in the coefficient table (nz + 4, level -2 first)
    long long si, sj;
};

// STEP: write phi + dt s (phi read exactly from set.in; the staged planes hold
// hi/lo pairs) at the column and at its periodic halo images
template <int NS, int TJ, bool BETA, int GMAX, bool STEP = false>
__global__ void __launch_bounds__(256)
pw_scalar_split_kernel(const __grid_constant__ CUtensorMap mu, const __grid_constant__ CUtensorMap mv,
                       const __grid_constant__ CUtensorMap mw, const __grid_constant__ PwScalarSplitSet set,
                       const float *__restrict__ cs, const PwScalarSplitGeom g, int *__restrict__ status,
                       double dt = 0.0) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if (pw_cta_failed(status)) return;
    // k chunks, then scalar groups, are the fastest grid indices: the chunks
    // and groups of one tile run together and share the wind planes in L2
    const int kchunk = blockIdx.x % g.nkc, grp = blockIdx.x / g.nkc;
    const int s0 = grp * g.group;
    const int G = min(g.group, g.n - s0);
    const int NF = 3 + G;
    const int fs = g.field_stride;
    const size_t slot_elems = (size_t)(3 + g.group) * fs;
    double *planes = reinterpret_cast<double *>(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + NS * slot_elems * 8);
    const int nt = blockDim.x, tid = threadIdx.x;
    const int nkt = g.kc / 2;
    const int tk = tid % nkt, tj = tid / nkt;
    const int j0 = blockIdx.y * TJ, i0 = blockIdx.z * g.ti, k0 = kchunk * g.kc;
    const int i_end = min(i0 + g.ti, g.nx);
    const int nplanes = i_end - i0 + 2;
    const uint32_t plane_bytes = (uint32_t)NF * (uint32_t)(TJ + 2) * (uint32_t)g.kb * 8u;
    const int kbase = k0 + 2 * tk, kk = 2 + 2 * tk, j = j0 + tj;

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
        double *dst = slot(p);
        pw_mbar_expect_tx(&bars[s], plane_bytes);
        const int c0 = k0 - 2, c1 = j0 + 1, c2 = i0 + 1 + p;
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
    auto wait = [&](int p) { return pw_mbar_wait_bounded(&bars[p % NS], (uint32_t)((p / NS) & 1)); };
    auto give_up = [&](int from) {
        if (tid == 0) {
            for (int p = from; p < issued; p++)
                if (!pw_mbar_wait_bounded(&bars[p % NS], (uint32_t)((p / NS) & 1), PW_DRAIN_CYCLES)) break;
            atomicExch(status, (int)PW_ERR_TIMEOUT);
        }
    };
    // in-place conversion of a landed plane, 16 bytes (two doubles) at a time,
    // from (x_k, x_k+1) to (hi_k, hi_k+1, lo_k, lo_k+1): thread (tk, tj) takes
    // chunk tk+1 of rows tj, tj+TJ, ...; the k-halo chunks 0 and nkt+1 of every
    // row are shared out over all threads
    const int rows = NF * (TJ + 2);
    bool bad = false;  // a value this thread converted was outside the split range
    auto conv_chunk = [&](double *base, int R, int c) {
        const int f = R / (TJ + 2), r = R - f * (TJ + 2);
        double *cp = base + (size_t)f * fs + (size_t)r * g.kb + 2 * c;
        const uint4 d = *reinterpret_cast<const uint4 *>(cp);
        // the winds (planes 0..2) and the scalars have their own ranges
        const uint32_t ehi = f < 3 ? PW_SPLIT_WIND_EHI : PW_SPLIT_SCALAR_EHI;
        float h0, l0, h1, l1;
        split_words(d.x, d.y, h0, l0, ehi, bad);
        split_words(d.z, d.w, h1, l1, ehi, bad);
        *reinterpret_cast<float4 *>(cp) = make_float4(h0, h1, l0, l1);
    };
    auto convert = [&](int p) {
        double *base = slot(p);
        for (int R = tj; R < rows; R += TJ) conv_chunk(base, R, tk + 1);
        for (int e = tid; e < 2 * rows; e += nt) conv_chunk(base, e >> 1, (e & 1) ? nkt + 1 : 0);
        pw_fence_proxy_async();  // the slot is refilled by TMA later
    };

    // coefficients of each level pair, prepared once per CTA in shared memory:
    // per pair t: g(k-1..k), g(k..k+1), 2 r(k..k+1); then hx, hy
    float4 *ctab = reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(bars) + 64);
    for (int t = tid; t < nkt; t += nt) {
        const int N = g.cs_n;
        const int kq = min(k0 + 2 * t, g.nz - 1);  // pairs past the top read valid entries
        const D2 c3[3] = {cs_pair(cs, N, 0, kq - 1), cs_pair(cs, N, 0, kq), cs_pair(cs, N, 2, kq)};
        for (int a = 0; a < 3; a++) {
            const float f = a == 2 ? 2.0f : 1.0f;  // doubling is exact
            ctab[t * 3 + a] = make_float4(f * lx(c3[a].h), f * ly(c3[a].h), f * lx(c3[a].l), f * ly(c3[a].l));
        }
    }
    if (tid == 0) {
        const float *tc = cs + 8 * g.cs_n;
        ctab[nkt * 3] = make_float4(2.0f * tc[0], 2.0f * tc[0], 2.0f * tc[1], 2.0f * tc[1]);
        ctab[nkt * 3 + 1] = make_float4(2.0f * tc[2], 2.0f * tc[2], 2.0f * tc[3], 2.0f * tc[3]);
    }
    auto coef = [&](int a) {
        const float4 c = ctab[tk * 3 + a];
        return D2{pk(c.x, c.y), pk(c.z, c.w)};
    };
    auto tcoef = [&](int a) {
        const float4 c = ctab[nkt * 3 + a];
        return D2{pk(c.x, c.y), pk(c.z, c.w)};
    };
    const bool active = (j < g.ny) && (kbase < g.nz);
    const int rS = tj * g.kb, rC = (tj + 1) * g.kb, rN = (tj + 2) * g.kb;

    // plane 0 (column i0-1): the x window of u and of each scalar
    D2 uM, pM[GMAX];
    {
        const bool ok = wait(0);
        if (ok) convert(0);
        if (!__syncthreads_and(ok)) {
            give_up(0);
            return;
        }
        const double *P0 = slot(0);
        uM = ld2<0>(P0 + rC, kk);
#pragma unroll
        for (int s = 0; s < GMAX; s++)
            if (s < G) pM[s] = ld2<0>(P0 + (size_t)(3 + s) * fs + rC, kk);
    }
    int waited = 1;
    for (int i = i0; i < i_end; i++) {
        const int q = i - i0 + 1;
        bool ok = true;
        while (ok && waited <= q + 1) {
            ok = wait(waited);
            if (ok) convert(waited++);
        }
        if (!__syncthreads_and(ok)) {
            give_up(waited);
            return;
        }
        // every thread is past step i-1 (planes q-1, q): refill the slot of q-1
        if (tid == 0 && q - 1 + NS < nplanes) {
            issue(q - 1 + NS);
            issued = q + NS;
        }
        const double *Pc = slot(q), *Pp = slot(q + 1);
        // wind factors shared by the scalars
        const D2 uC = ld2<0>(Pc + rC, kk);
        const D2 hx = tcoef(0), hy = tcoef(1);
        const D2 HUm = df_mul(uM, hx), HUc = df_mul(uC, hx);
        const D2 HVs = df_mul(ld2<0>(Pc + fs + rS, kk), hy), HVc = df_mul(ld2<0>(Pc + fs + rC, kk), hy);
        const double *wr = Pc + 2 * fs + rC;
        const D2 r2 = coef(2);
        const D2 A = df_mul(df_mul(ld2<-1>(wr, kk), coef(0)), r2);
        const D2 B = df_mul(df_mul(ld2<0>(wr, kk), coef(1)), r2);
        const long long off = (long long)(i + 2) * g.si + (long long)(j + 2) * g.sj + kbase;
#pragma unroll
        for (int s = 0; s < GMAX; s++) {
            if (s < G) {
                const double *pr = Pc + (size_t)(3 + s) * fs;
                const D2 pC = ld2<0>(pr + rC, kk);
                if (active) {
                    const D2 X = df_sub(df_mul(HUm, pM[s]), df_mul(HUc, ld2<0>(Pp + (size_t)(3 + s) * fs + rC, kk)));
                    const D2 Y = df_sub(df_mul(HVs, ld2<0>(pr + rS, kk)), df_mul(HVc, ld2<0>(pr + rN, kk)));
                    const D2 Z = df_sub(df_mul(A, ld2<-1>(pr + rC, kk)), df_mul(B, ld2<1>(pr + rC, kk)));
                    const D2 r = df_add(df_add(X, Y), Z);
                    double a0 = join(lx(r.h), lx(r.l)), a1 = join(ly(r.h), ly(r.l));
                    if constexpr (STEP) {
                        const double *px = set.in[s0 + s] + off;
                        const bool two = kbase + 1 < g.nz;
                        const double o2[2] = {fma(dt, a0, px[0]), two ? fma(dt, a1, px[1]) : 0.0};
                        pw_store_images<double, 2>(set.out[s0 + s], i, j, kbase, o2, g.nz - kbase, g.nx, g.ny,
                                                   g.si, g.sj);
                    } else {
                        double *po = set.out[s0 + s] + off;
                        if (kbase + 1 < g.nz) {
                            if (BETA) {
                                const double2 o = *reinterpret_cast<const double2 *>(po);
                                a0 += o.x;
                                a1 += o.y;
                            }
                            *reinterpret_cast<double2 *>(po) = make_double2(a0, a1);
                        } else {
                            po[0] = BETA ? po[0] + a0 : a0;
                        }
                    }
                }
                pM[s] = pC;
            }
        }
        uM = uC;
    }
    if (__syncthreads_or(bad) && tid == 0) atomicOr(status + PW_STATUS_RANGE_WORD, 1);
    if (tid == 0)
        for (int s = 0; s < NS; s++) pw_mbar_inval(&bars[s]);
}

pw_status pw_launch_scalars_split(const pw_mesh *m, const void *u, const void *v, const void *w, int n,
                                  const void *const *phi, void *const *sphi, int beta, cudaStream_t st,
                                  int tile_j, int tile_i, int group, bool step, double dt) {
    constexpr int NS = PW_SSPLIT_NS;
    // compiled for 4 or 8 rows of columns per CTA (the nearest of the two is used)
    tile_j = tile_j <= 5 ? 4 : 8;
    PwScalarSplitGeom g;
    g.nx = m->nx;
    g.ny = m->ny;
    g.nz = m->nz;
    const int kc_one = (m->nz + 1) / 2 * 2, kc_max = tile_j == 4 ? 64 : 32;  // 128 threads per CTA
    g.kc = kc_one <= kc_max ? kc_one : kc_max;
    g.kb = g.kc + 4;
    const int plane_elems = (tile_j + 2) * g.kb;
    g.field_stride = (plane_elems + 15) / 16 * 16;  // 128-byte aligned planes
    g.cs_n = m->nz + 4;
    g.si = m->si;
    g.sj = m->sj;
    const int threads = (g.kc / 2) * tile_j;
    if (threads > 256)
        return pw_fail(PW_ERR_SHAPE, "scalar split kernel: tile_j=%d needs %d threads (max 256)", tile_j, threads);
    static_assert(PW_SSPLIT_NS * sizeof(uint64_t) <= 64, "barrier slot");
    const size_t field_bytes = (size_t)NS * g.field_stride * 8;
    const size_t fixed = 64 + ((size_t)(g.kc / 2) * 3 + 2) * sizeof(float4);
    if (group <= 0) {
        // the largest group whose CTA still lets 4 CTAs share an SM (228 KB of
        // shared memory, 1 KB of it reserved per CTA): the double-float arithmetic
        // needs the warps to hide its latency, so two groups of three scalars at 16
        // warps per SM beat one group of six at 8 (148 vs 129 G values/s for
        // theta + 5 q on 1024 x 1024 x 128) although the wind is staged twice
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
        pw_status s = pw_make_field_map(&maps[q], f[q], PW_F64, m->nx, m->ny, m->nzp, pw_kdim(m->nz, q), g.kb,
                                        tile_j + 2);
        if (s != PW_OK) return s;
    }
    PwScalarSplitSet set;
    memset(&set, 0, sizeof(set));
    for (int q = 0; q < n; q++) {
        pw_status s = pw_make_field_map(&set.phi[q], phi[q], PW_F64, m->nx, m->ny, m->nzp, m->nz, g.kb,
                                        tile_j + 2);
        if (s != PW_OK) return s;
        set.out[q] = (double *)sphi[q];
        set.in[q] = (const double *)phi[q];
    }
    constexpr int GM = PW_SSPLIT_GMAX;
    auto kern = step ? (tile_j == 4 ? pw_scalar_split_kernel<NS, 4, false, GM, true>
                                    : pw_scalar_split_kernel<NS, 8, false, GM, true>)
                     : tile_j == 4 ? (beta ? pw_scalar_split_kernel<NS, 4, true, GM> : pw_scalar_split_kernel<NS, 4, false, GM>)
                                   : (beta ? pw_scalar_split_kernel<NS, 8, true, GM> : pw_scalar_split_kernel<NS, 8, false, GM>);
    PW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long ngroups = (n + group - 1) / group;
    // the wave rule of pw_pick_tile_i measured slower here (a longer march for
    // 149 -> 140 G values/s on theta + 5 q, 1024 x 1024 x 128), so the grid keeps
    // the fill rule
    tile_i = pw_fit_tile_i(m, tile_i, (long)((m->ny + tile_j - 1) / tile_j) * g.nkc);
    g.ti = tile_i;
    dim3 grid((unsigned)(g.nkc * ngroups), (unsigned)((m->ny + tile_j - 1) / tile_j),
              (unsigned)((m->nx + tile_i - 1) / tile_i));
    if (grid.y > 65535 || grid.z > 65535) return pw_fail(PW_ERR_SHAPE, "grid too large; raise tile_j or tile_i");
    kern<<<grid, threads, smem, st>>>(maps[0], maps[1], maps[2], set, m->coefsplit, g, m->status, dt);
    PW_CUDA(cudaGetLastError());
    return PW_OK;
}
