// pw_march.cuh -- the x-march over TMA-staged (j,k) planes, shared by the
// single-mesh stencil kernel (pw_advect.cu) and the persistent batched kernel
// (pw_batch.cu).
//
// Each thread owns KV consecutive levels of one column and a warp covers a
// whole column segment with 16-byte accesses.  A CTA tile is tile_j rows of
// columns (y) and one k chunk, marched along x: a ring of ns (j,k) planes of
// u, v, w lives in shared memory, each holding tile_j + 2 rows (the y halo)
// and the k chunk plus a 16-byte k halo on each side.  Planes are fetched by
// TMA (one elected thread, completion on an mbarrier) ns - 3 planes ahead of
// the one being consumed, so every value of u, v, w is read from HBM once per
// tile (plus the y halo and the two priming planes).  Each step computes su,
// sv, sw for plane i from planes i-1, i, i+1 and stores them with 16-byte
// stores.
#pragma once

#include <type_traits>

#include "pw_internal.h"

// planes in the shared-memory ring of the x-march (NS - 3 planes of prefetch)
#define PW_MARCH_NS 5

struct PwGeom {
    int nx, ny, nz, nzp;
    int kc;            // k chunk per CTA (multiple of KV and of the k halo)
    int kb;            // TMA box k extent = kc + 2*h
    int h;             // k halo in elements (16 bytes)
    int tj, ti;        // rows per CTA, columns marched per CTA
    int ns;            // planes in the ring
    int field_stride;  // elements between the u, v, w planes of one slot
    int plane_elems;   // (tj + 2) * kb
    long long si, sj;  // strides of the sources (elements)
    double tcx, tcy;
    float ftcx, ftcy;  // the same rounded to FP32 on the host (the FP32 kernels take these)
};

// a host-supplied constant in the compute type: FP32 kernels take the FP32
// copy, so no thread spends FP64 conversions on it
template <typename TC>
__device__ __forceinline__ TC pw_geom_c(double d, float f) {
    if constexpr (std::is_same<TC, float>::value) return f;
    else return (TC)d;
}

// --------------------------------------------------------------------------
// slab loads from shared memory: KV values at [kk, kk+KV) plus optional
// neighbours kk-1 and kk+KV, widened to the compute type
// --------------------------------------------------------------------------
template <typename TS, typename TC, int KV>
struct SlabLoad;

template <typename TC>
struct SlabLoad<float, TC, 4> {
    static __device__ __forceinline__ void run(const float *p, TC *o) {
        float4 a = *reinterpret_cast<const float4 *>(p);
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    }
};
template <typename TC>
struct SlabLoad<double, TC, 2> {
    static __device__ __forceinline__ void run(const double *p, TC *o) {
        double2 a = *reinterpret_cast<const double2 *>(p);
        o[0] = a.x; o[1] = a.y;
    }
};
template <typename TC>
struct SlabLoad<double, TC, 4> {
    static __device__ __forceinline__ void run(const double *p, TC *o) {
        double2 a = *reinterpret_cast<const double2 *>(p);
        double2 b = *reinterpret_cast<const double2 *>(p + 2);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
};
template <typename TC>
struct SlabLoad<__nv_bfloat16, TC, 4> {
    static __device__ __forceinline__ void run(const __nv_bfloat16 *p, TC *o) {
        uint2 a = *reinterpret_cast<const uint2 *>(p);
        // bf16 -> f32 is exact: the bf16 bits are the top half of the f32
        o[0] = __uint_as_float(a.x << 16);
        o[1] = __uint_as_float(a.x & 0xffff0000u);
        o[2] = __uint_as_float(a.y << 16);
        o[3] = __uint_as_float(a.y & 0xffff0000u);
    }
};

// x[0] = value at k-1, x[1..KV] = k..k+KV-1, x[KV+1] = k+KV
template <typename TS, typename TC, int KV, bool LO, bool HI>
__device__ __forceinline__ void pw_col(const TS *row, int kk, TC (&x)[KV + 2]) {
    SlabLoad<TS, TC, KV>::run(row + kk, x + 1);
    x[0] = LO ? pw_to<TC>(row[kk - 1]) : TC(0);
    x[KV + 1] = HI ? pw_to<TC>(row[kk + KV]) : TC(0);
}

// --------------------------------------------------------------------------
// vector stores of KV results (with optional accumulate), masked at the top
// --------------------------------------------------------------------------
template <typename TO, int KV>
__device__ __forceinline__ void pw_store(TO *p, const TO (&r)[KV], int nvalid, int beta) {
    if (nvalid >= KV) {
        if constexpr (sizeof(TO) * KV == 16) {
            using V = typename std::conditional<sizeof(TO) == 8, double2, float4>::type;
            V val;
            TO *vv = reinterpret_cast<TO *>(&val);
            if (beta) {
                V old = *reinterpret_cast<const V *>(p);
                const TO *oo = reinterpret_cast<const TO *>(&old);
#pragma unroll
                for (int m = 0; m < KV; m++) vv[m] = oo[m] + r[m];
            } else {
#pragma unroll
                for (int m = 0; m < KV; m++) vv[m] = r[m];
            }
            *reinterpret_cast<V *>(p) = val;
        } else if constexpr (sizeof(TO) * KV == 8) {
            // four bfloat16 results: one 8-byte store (accumulation in FP32,
            // rounded once)
            struct alignas(8) V8 {
                TO v[KV];
            };
            V8 val;
            if (beta) {
                const V8 old = *reinterpret_cast<const V8 *>(p);
#pragma unroll
                for (int m = 0; m < KV; m++) val.v[m] = (TO)(pw_to<float>(old.v[m]) + pw_to<float>(r[m]));
            } else {
#pragma unroll
                for (int m = 0; m < KV; m++) val.v[m] = r[m];
            }
            *reinterpret_cast<V8 *>(p) = val;
        } else {
#pragma unroll
            for (int m = 0; m < KV; m++) p[m] = beta ? TO(p[m] + r[m]) : r[m];
        }
    } else {
        // the top of the column: the stored values are read only when accumulating
        if (beta) {
#pragma unroll
            for (int m = 0; m < KV; m++)
                if (m < nvalid) p[m] = p[m] + r[m];
        } else {
#pragma unroll
            for (int m = 0; m < KV; m++)
                if (m < nvalid) p[m] = r[m];
        }
    }
}

// --------------------------------------------------------------------------
// k edges of a thread's slab: the value below comes from the thread holding the
// previous slab of the same column (one lane down), the value above from the
// next slab's thread (one lane up), by warp shuffles; threads at the ends of a
// column (or of a warp) read those values from shared memory instead.
// --------------------------------------------------------------------------
template <typename TS, typename TC, int KV>
__device__ __forceinline__ void pw_col_edges(const TS *row, int kk, TC (&x)[KV + 2], unsigned mask,
                                             bool lo_shfl, bool hi_shfl, bool want_lo, bool want_hi) {
    SlabLoad<TS, TC, KV>::run(row + kk, x + 1);
    if (want_lo) {
        const TC up = __shfl_up_sync(mask, x[KV], 1);
        if (lo_shfl) x[0] = up;
        else x[0] = pw_to<TC>(row[kk - 1]);
    } else {
        x[0] = TC(0);
    }
    if (want_hi) {
        const TC dn = __shfl_down_sync(mask, x[1], 1);
        if (hi_shfl) x[KV + 1] = dn;
        else x[KV + 1] = pw_to<TC>(row[kk + KV]);
    } else {
        x[KV + 1] = TC(0);
    }
}

template <typename TC, int KV>
__device__ __forceinline__ void pw_copy(TC (&d)[KV + 2], const TC (&s)[KV + 2]) {
#pragma unroll
    for (int m = 0; m < KV + 2; m++) d[m] = s[m];
}

// --------------------------------------------------------------------------
// store KV values of interior column (i, j) at the column and at every halo
// column that is its periodic image (halo coordinates ih, jh in [0, n+4))
// --------------------------------------------------------------------------
template <typename TO, int KV>
__device__ __forceinline__ void pw_store_images(TO *base, int i, int j, int kbase, const TO (&r)[KV],
                                                int nvalid, int nx, int ny, long long si, long long sj) {
    pw_store<TO, KV>(base + (long long)(i + 2) * si + (long long)(j + 2) * sj + kbase, r, nvalid, 0);
    if (i >= 2 && i < nx - 2 && j >= 2 && j < ny - 2) return;
    for (int ih = i + 2 - ((i + 2) / nx) * nx; ih < nx + 4; ih += nx)
        for (int jh = j + 2 - ((j + 2) / ny) * ny; jh < ny + 4; jh += ny) {
            if (ih >= 2 && ih < nx + 2 && jh >= 2 && jh < ny + 2) continue;  // the interior column
            pw_store<TO, KV>(base + (long long)ih * si + (long long)jh * sj + kbase, r, nvalid, 0);
        }
}

// --------------------------------------------------------------------------
// one tile of the x-march: tile_j rows from j0, columns i0 .. i0+tile_i-1, the
// k chunk starting at k0.  Shared memory: NS plane slots then NS mbarriers
// (initialised here, invalidated before returning so the caller may run the
// next tile).  Returns false if a TMA wait timed out (status recorded).
//
// Register window along x: the centre-row columns of planes i-1 and i and the
// side rows' values that the next step needs are carried in registers, so a
// step loads only column i+1 of the centre row and the rows j-1, j+1 it still
// lacks (9 slabs and 8 edge values instead of 17 slabs and 9 edges).  Levels
// at or above nz (and the w lid) arrive from TMA as zeros: the tensor maps
// carry the logical k extent.
// --------------------------------------------------------------------------
//
// STEP: instead of the sources, write x + dt S(x) for x = u, v, w (the forward
// Euler step fused into the stencil: x is the centre value already in
// registers) to su, sv, sw, which then have the field type, at the interior
// column and at its periodic halo images (ready for the next step).
template <typename TS, typename TC, typename TO, int KV, int NS, bool STEP = false>
__device__ __forceinline__ bool pw_march_tile(const CUtensorMap *mu_, const CUtensorMap *mv_,
                                              const CUtensorMap *mw_, TO *__restrict__ su,
                                              TO *__restrict__ sv, TO *__restrict__ sw,
                                              const TC *__restrict__ coef, const PwGeom &g, int beta,
                                              int *__restrict__ status, unsigned char *smem_raw,
                                              int j0, int i0, int k0, double dt = 0.0) {
    const CUtensorMap &mu = *mu_, &mv = *mv_, &mw = *mw_;
    TS *planes = reinterpret_cast<TS *>(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + (size_t)NS * 3 * g.field_stride * sizeof(TS));
    const int fs = g.field_stride;

    const int nkt = g.kc / KV;
    const int tid = threadIdx.x, lane = tid & 31;
    const int tk = tid % nkt, tj = tid / nkt;
    const int i_end = min(i0 + g.ti, g.nx);
    const int nplanes = i_end - i0 + 2;  // planes i0-1 .. i_end
    const uint32_t plane_bytes = 3u * (uint32_t)g.plane_elems * (uint32_t)sizeof(TS);
    const int kbase = k0 + tk * KV;      // first level of this thread
    const int kk = g.h + tk * KV;        // its position inside a plane row
    const int j = j0 + tj;
    const bool in_tile = tj < g.tj;
    const int tjc = in_tile ? tj : g.tj - 1;  // rows read by threads outside the tile stay in the plane
    const bool active = in_tile && (j < g.ny) && (kbase < g.nz);
    const int nvalid = g.nz - kbase;
    // shuffle partners: same column, same warp; lanes of a partial last warp
    const int wbase = tid & ~31;
    const unsigned mask = (int)blockDim.x - wbase >= 32 ? 0xffffffffu
                                                         : ((1u << ((int)blockDim.x - wbase)) - 1u);
    const bool lo_shfl = tk > 0 && lane > 0;
    const bool hi_shfl = tk < nkt - 1 && lane < 31 && tid + 1 < (int)blockDim.x;

    if (threadIdx.x == 0) {
        pw_prefetch_map(&mu);
        pw_prefetch_map(&mv);
        pw_prefetch_map(&mw);
        for (int s = 0; s < NS; s++) pw_mbar_init(&bars[s], 1);
        pw_fence_barrier_init();
    }
    __syncthreads();

    auto issue = [&](int p) {
        const int s = p % NS;
        TS *dst = planes + (size_t)s * 3 * fs;
        pw_mbar_expect_tx(&bars[s], plane_bytes);
        const int c0 = k0 - g.h, c1 = j0 + 1, c2 = i0 + 1 + p;  // (k, j-1, i-1+p) + halo offset
        pw_tma_load_3d(dst, &mu, c0, c1, c2, &bars[s]);
        pw_tma_load_3d(dst + fs, &mv, c0, c1, c2, &bars[s]);
        pw_tma_load_3d(dst + 2 * fs, &mw, c0, c1, c2, &bars[s]);
    };
    int issued = 0;  // planes handed to TMA (thread 0's count)
    if (threadIdx.x == 0) {
        for (int p = 0; p < min(NS, nplanes); p++) issue(p);
        issued = min(NS, nplanes);
    }
    auto slot = [&](int p) { return planes + (size_t)(p % NS) * 3 * fs; };
    auto give_up = [&](int waited) {
        if (threadIdx.x == 0) {
            for (int p = waited; p < issued; p++)
                if (!pw_mbar_wait_bounded(&bars[p % NS], (uint32_t)((p / NS) & 1), PW_DRAIN_CYCLES)) break;
            atomicExch(status, (int)PW_ERR_TIMEOUT);
        }
    };

    // vertical coefficients of this thread's levels (0 beyond nz)
    TC c1[KV], c2[KV], d1[KV], d2[KV];
#pragma unroll
    for (int m = 0; m < KV; m++) {
        const int k = kbase + m;
        const bool in = k < g.nz;
        c1[m] = in ? coef[k] : TC(0);
        c2[m] = in ? coef[g.nz + k] : TC(0);
        d1[m] = in ? coef[2 * g.nz + k] : TC(0);
        d2[m] = in ? coef[3 * g.nz + k] : TC(0);
    }
    const TC tcx = pw_geom_c<TC>(g.tcx, g.ftcx), tcy = pw_geom_c<TC>(g.tcy, g.ftcy);
    const TC tdt = (TC)dt;
    const int L = g.kb;
    const int rS = tjc * L, rC = (tjc + 1) * L, rN = (tjc + 2) * L;

    // the window: planes 0 (column i0-1) and 1 (column i0)
    TC uM[KV + 2], uC[KV + 2], vM[KV + 2], vC[KV + 2], wM[KV + 2], wC[KV + 2], vS[KV + 2], uNM[KV + 2];
    {
        const bool ok = pw_mbar_wait_bounded(&bars[0], 0) && pw_mbar_wait_bounded(&bars[1], 0);
        if (!__syncthreads_and(ok)) {
            give_up(0);
            return false;
        }
        const TS *P0 = slot(0), *P1 = slot(1);
        pw_col_edges<TS, TC, KV>(P0 + rC, kk, uM, mask, lo_shfl, hi_shfl, false, true);
        pw_col_edges<TS, TC, KV>(P1 + rC, kk, uC, mask, lo_shfl, hi_shfl, true, true);
        pw_col_edges<TS, TC, KV>(P0 + fs + rC, kk, vM, mask, lo_shfl, hi_shfl, false, false);
        pw_col_edges<TS, TC, KV>(P1 + fs + rC, kk, vC, mask, lo_shfl, hi_shfl, true, true);
        pw_col_edges<TS, TC, KV>(P0 + 2 * fs + rC, kk, wM, mask, lo_shfl, hi_shfl, false, false);
        pw_col_edges<TS, TC, KV>(P1 + 2 * fs + rC, kk, wC, mask, lo_shfl, hi_shfl, true, true);
        pw_col_edges<TS, TC, KV>(P1 + fs + rS, kk, vS, mask, lo_shfl, hi_shfl, false, true);
        pw_col_edges<TS, TC, KV>(P0 + rN, kk, uNM, mask, lo_shfl, hi_shfl, false, false);
    }

    int waited = 2;
    for (int i = i0; i < i_end; i++) {
        const int q = i - i0 + 1;  // plane index of column i
        bool ok = true;
        if (waited <= q + 1) {
            ok = pw_mbar_wait_bounded(&bars[(q + 1) % NS], (uint32_t)(((q + 1) / NS) & 1));
            if (ok) waited = q + 2;
        }
        if (!__syncthreads_and(ok)) {
            give_up(waited);
            return false;
        }
        // everyone is past step i-1: the slot of plane q-2 is free
        if (threadIdx.x == 0 && q >= 2 && q - 2 + NS < nplanes) {
            issue(q - 2 + NS);
            issued = q - 1 + NS;
        }
        const TS *Pc = slot(q), *Pp = slot(q + 1);

        TC uP[KV + 2], vP[KV + 2], wP[KV + 2], uS[KV + 2], wS[KV + 2], vSP[KV + 2];
        TC uN[KV + 2], vN[KV + 2], wN[KV + 2];
        pw_col_edges<TS, TC, KV>(Pp + rC, kk, uP, mask, lo_shfl, hi_shfl, true, true);
        pw_col_edges<TS, TC, KV>(Pp + fs + rC, kk, vP, mask, lo_shfl, hi_shfl, true, true);
        pw_col_edges<TS, TC, KV>(Pp + 2 * fs + rC, kk, wP, mask, lo_shfl, hi_shfl, true, true);
        pw_col_edges<TS, TC, KV>(Pc + rS, kk, uS, mask, lo_shfl, hi_shfl, false, false);
        pw_col_edges<TS, TC, KV>(Pc + 2 * fs + rS, kk, wS, mask, lo_shfl, hi_shfl, false, false);
        pw_col_edges<TS, TC, KV>(Pp + fs + rS, kk, vSP, mask, lo_shfl, hi_shfl, false, true);
        pw_col_edges<TS, TC, KV>(Pc + rN, kk, uN, mask, lo_shfl, hi_shfl, false, false);
        pw_col_edges<TS, TC, KV>(Pc + fs + rN, kk, vN, mask, lo_shfl, hi_shfl, false, false);
        pw_col_edges<TS, TC, KV>(Pc + 2 * fs + rN, kk, wN, mask, lo_shfl, hi_shfl, true, false);
        if (active) {
            TO ru[KV], rv[KV], rw[KV];
#pragma unroll
            for (int m = 0; m < KV; m++) {
                const int a = m + 1;  // index of level kbase+m in the slab arrays
                TC s;
                s = tcx * (uM[a] * (uM[a] + uC[a]) - uP[a] * (uC[a] + uP[a]));
                s = s + tcy * (uS[a] * (vS[a] + vSP[a]) - uN[a] * (vC[a] + vP[a]));
                s = s + c1[m] * uC[a - 1] * (wC[a - 1] + wP[a - 1]);
                s = s - c2[m] * uC[a + 1] * (wC[a] + wP[a]);
                ru[m] = STEP ? (TO)(uC[a] + tdt * s) : (TO)s;
                s = tcx * (vM[a] * (uM[a] + uNM[a]) - vP[a] * (uC[a] + uN[a]));
                s = s + tcy * (vS[a] * (vS[a] + vC[a]) - vN[a] * (vC[a] + vN[a]));
                s = s + c1[m] * vC[a - 1] * (wC[a - 1] + wN[a - 1]);
                s = s - c2[m] * vC[a + 1] * (wC[a] + wN[a]);
                rv[m] = STEP ? (TO)(vC[a] + tdt * s) : (TO)s;
                s = tcx * (wM[a] * (uM[a] + uM[a + 1]) - wP[a] * (uC[a] + uC[a + 1]));
                s = s + tcy * (wS[a] * (vS[a] + vS[a + 1]) - wN[a] * (vC[a] + vC[a + 1]));
                s = s + d1[m] * wC[a - 1] * (wC[a - 1] + wC[a]);
                s = s - d2[m] * wC[a + 1] * (wC[a] + wC[a + 1]);
                // the lid level of w reads as 0, so a step leaves it 0
                rw[m] = (kbase + m < g.nz - 1) ? (STEP ? (TO)(wC[a] + tdt * s) : (TO)s) : TO(0);
            }
            if (STEP) {
                pw_store_images<TO, KV>(su, i, j, kbase, ru, nvalid, g.nx, g.ny, g.si, g.sj);
                pw_store_images<TO, KV>(sv, i, j, kbase, rv, nvalid, g.nx, g.ny, g.si, g.sj);
                pw_store_images<TO, KV>(sw, i, j, kbase, rw, nvalid, g.nx, g.ny, g.si, g.sj);
            } else {
                const long long off = (long long)(i + 2) * g.si + (long long)(j + 2) * g.sj + kbase;
                pw_store<TO, KV>(su + off, ru, nvalid, beta);
                pw_store<TO, KV>(sv + off, rv, nvalid, beta);
                pw_store<TO, KV>(sw + off, rw, nvalid, beta);
            }
        }
        // slide the window one column along x
        pw_copy<TC, KV>(uM, uC);
        pw_copy<TC, KV>(uC, uP);
        pw_copy<TC, KV>(vM, vC);
        pw_copy<TC, KV>(vC, vP);
        pw_copy<TC, KV>(wM, wC);
        pw_copy<TC, KV>(wC, wP);
        pw_copy<TC, KV>(vS, vSP);
        pw_copy<TC, KV>(uNM, uN);
    }
    __syncthreads();  // every thread is past its last wait: barriers can be reused
    if (threadIdx.x == 0)
        for (int s = 0; s < NS; s++) pw_mbar_inval(&bars[s]);
    __syncthreads();
    return true;
}
