// pw_residuals.cu -- the FP64 conservation sums (A5): for each component
// phi in (u, v, w) with source S and energy weight W (rho_n dz on u/v levels,
// rho_w dzn on w faces, 0 on the lid face),
//   sum W phi S,  sum W |phi S|,  sum W S,  sum W |S|
// over the interior, in a deterministic tree reduction (a fixed grid, a fixed
// order of terms per thread, a fixed tree per block, and the block records
// added in a fixed order by whichever block finishes last), so repeated calls
// give the same bits.
//
// The fast pass keeps FP64 accuracy without the FP64 units (which run at
// ~1/80 of the FP32 rate on B300): every value is split with integer bit
// operations into a (hi, lo) pair of floats, the products phi S are formed with
// FMA-exact transforms and each thread accumulates double-float sums on the
// FP32 pipe (packed .f32x2 over the two levels it owns).  A warp owns one block
// of 64 levels of every column of its column group, so a thread always adds
// terms of the same two levels and applies their weights once, in FP64, at the
// end.  The relative error of each sum is a few units of 2^-46 of the sum of
// the magnitudes of its terms.  Values it cannot carry exactly (a nonzero
// |x| < 2^-100, |x| >= 2^56, NaN or Inf) are counted, and so are sums of
// magnitudes below 2^-40; then the sums are recomputed by the plain FP64 pass.
#include "pw_df.cuh"
#include "pw_internal.h"

// Unscaled split of a double (words xl, xh) into hi (24 leading significant
// bits) + lo (the next 23): exact to 2^-46 relative for 2^-100 <= |x| < 2^56;
// other nonzero values give (0, 0) and set `bad`.
__device__ __forceinline__ void pw_res_split(uint32_t xl, uint32_t xh, float &hi, float &lo, bool &bad) {
    const uint32_t f = __funnelshift_l(xl, xh, 3) + 0x40000000u;  // exponent 1023 -> 127
    const uint32_t hb = (f & 0x7fffffffu) | (xh & 0x80000000u);
    const uint32_t cb = (hb & 0xff800000u) - 0x0b800000u;
    const uint32_t fb = cb | ((xl >> 6) & 0x007fffffu);
    const uint32_t e = xh & 0x7ff00000u;
    const bool inr = (e - (923u << 20)) < ((1079u - 923u) << 20);
    bad |= !inr && ((xh & 0x7fffffffu) | xl) != 0u;
    hi = inr ? __uint_as_float(hb) : 0.0f;
    lo = inr ? __uint_as_float(fb) - __uint_as_float(cb) : 0.0f;
}
// the same range test for a float value (exact as hi, lo = 0)
__device__ __forceinline__ float pw_res_float(float x, bool &bad) {
    const uint32_t b = __float_as_uint(x) & 0x7fffffffu;
    const bool inr = b >= 0x0d800000u && b < 0x5b800000u;  // [2^-100, 2^56)
    bad |= !inr && b != 0u;
    return inr ? x : 0.0f;
}

// hi + lo as a double (one FP64 add); zeros and subnormal floats give 0
__device__ __forceinline__ double pw_res_join(float hi, float lo) {
    const double h = (__float_as_uint(hi) & 0x7f800000u) ? (double)hi : 0.0;
    const double l = (__float_as_uint(lo) & 0x7f800000u) ? (double)lo : 0.0;
    return h + l;
}

// The two levels (k, k+1) of one column of a field: `raw` loads them (one
// vector load) and `run` makes the double-float pair; levels outside the
// field (ok0, ok1 false) read as 0.
template <typename T>
struct PwResLoad;
template <>
struct PwResLoad<double> {
    using Raw = uint4;
    static __device__ __forceinline__ Raw raw(const double *p) { return *reinterpret_cast<const uint4 *>(p); }
    static __device__ __forceinline__ D2 run(Raw d, bool ok0, bool ok1, bool &bad) {
        float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
        if (ok0) pw_res_split(d.x, d.y, h0, l0, bad);
        if (ok1) pw_res_split(d.z, d.w, h1, l1, bad);
        return D2{pk(h0, h1), pk(l0, l1)};
    }
};
template <>
struct PwResLoad<float> {
    using Raw = float2;
    static __device__ __forceinline__ Raw raw(const float *p) { return *reinterpret_cast<const float2 *>(p); }
    static __device__ __forceinline__ D2 run(Raw d, bool ok0, bool ok1, bool &bad) {
        const float a = ok0 ? pw_res_float(d.x, bad) : 0.f, b = ok1 ? pw_res_float(d.y, bad) : 0.f;
        return D2{pk(a, b), pk(0.f, 0.f)};
    }
};
template <>
struct PwResLoad<__nv_bfloat16> {
    using Raw = uint32_t;
    static __device__ __forceinline__ Raw raw(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }
    static __device__ __forceinline__ D2 run(Raw d, bool ok0, bool ok1, bool &bad) {
        const float a = ok0 ? pw_res_float(__uint_as_float(d << 16), bad) : 0.f;
        const float b = ok1 ? pw_res_float(__uint_as_float(d & 0xffff0000u), bad) : 0.f;
        return D2{pk(a, b), pk(0.f, 0.f)};
    }
};

// |x| of each lane of a double-float pair (the sign of a lane is its hi's)
__device__ __forceinline__ D2 pw_res_abs(D2 x) {
    const unsigned long long m = x.h.v & 0x8000000080000000ull;
    return D2{P2{x.h.v ^ m}, P2{x.l.v ^ m}};
}

// fixed-order tree over the block: vals[PW_RED_STRIDE] of every thread -> out
template <int NT>
__device__ __forceinline__ void pw_res_block_tree(double (&vals)[PW_RED_STRIDE], double *out) {
    __shared__ double red[PW_RED_STRIDE][NT];
#pragma unroll
    for (int q = 0; q < PW_RED_STRIDE; q++) red[q][threadIdx.x] = vals[q];
    __syncthreads();
    for (int h = NT / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int q = 0; q < PW_RED_STRIDE; q++) red[q][threadIdx.x] += red[q][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < PW_RED_STRIDE) out[threadIdx.x] = red[threadIdx.x][0];
}

// After a block's record is written: the last block to finish adds the
// PW_RED_BLOCKS records (thread t: records t, t + NT, ..., all loads issued
// before the first add), then the fixed tree, into the totals, and sets the
// counter back to 0.  Which block is last does not change the order.
template <int NT>
__device__ __forceinline__ void pw_res_finish(double *scratch) {
    constexpr int PER = (PW_RED_BLOCKS + NT - 1) / NT;
    __shared__ unsigned ticket;
    __threadfence();  // this block's record is visible before its ticket
    __syncthreads();
    unsigned *count = reinterpret_cast<unsigned *>(scratch + PW_RED_SCRATCH - 1);
    if (threadIdx.x == 0) ticket = atomicAdd(count, 1u);
    __syncthreads();
    if (ticket != PW_RED_BLOCKS - 1) return;
    __threadfence();
    double r[PER][PW_RED_STRIDE];
#pragma unroll
    for (int m = 0; m < PER; m++) {
        const int b = (int)threadIdx.x + m * NT;
#pragma unroll
        for (int q = 0; q < PW_RED_STRIDE; q++) r[m][q] = b < PW_RED_BLOCKS ? __ldcg(scratch + (size_t)b * PW_RED_STRIDE + q) : 0.0;
    }
    double vals[PW_RED_STRIDE];
#pragma unroll
    for (int q = 0; q < PW_RED_STRIDE; q++) {
        double a = r[0][q];
#pragma unroll
        for (int m = 1; m < PER; m++) a += r[m][q];
        vals[q] = a;
    }
    pw_res_block_tree<NT>(vals, scratch + PW_RED_BLOCKS * PW_RED_STRIDE);
    if (threadIdx.x == 0) *count = 0u;
}

template <typename TF, typename TS>
__global__ void __launch_bounds__(PW_RED_FAST_THREADS)
pw_residual_fast(const TF *u, const TF *v, const TF *w, const TS *su, const TS *sv, const TS *sw,
                 const double *wuv, const double *ww, int nx, int ny, int nz, int nzp,
                 double *partials) {
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    const int nkb = (nz + 63) / 64;       // blocks of 64 levels
    const int ngrp = nw / nkb;            // column groups (warps past ngrp * nkb idle)
    const int kblk = gw % nkb, grp = gw / nkb;
    const int k = kblk * 64 + 2 * lane;   // this thread's levels k, k+1
    const bool ok0 = k < nz, ok1 = k + 1 < nz;
    const bool okw0 = k < nz - 1, okw1 = k + 1 < nz - 1;  // w faces below the lid
    const D2 zero{P2{0ull}, P2{0ull}};
    D2 acc[12];
#pragma unroll
    for (int q = 0; q < 12; q++) acc[q] = zero;
    bool bad = false;
    if (grp < ngrp && grp < nx * ny && ok0) {
        using LF = PwResLoad<TF>;
        using LS = PwResLoad<TS>;
        // columns grp, grp + ngrp, ...: (i, j) stepped without divisions, and
        // the next column's values loaded before this column's arithmetic (two
        // columns of loads in flight per thread)
        const int ncol = nx * ny, di = ngrp / ny, dj = ngrp - di * ny;
        int c = grp, i = grp / ny, j = grp - (grp / ny) * ny;
        auto at = [&](int ii, int jj) { return ((long long)(ii + 2) * (ny + 4) + (jj + 2)) * nzp + k; };
        long long off = at(i, j);
        typename LF::Raw fr[3] = {LF::raw(u + off), LF::raw(v + off), LF::raw(w + off)};
        typename LS::Raw sr[3] = {LS::raw(su + off), LS::raw(sv + off), LS::raw(sw + off)};
        while (true) {
            const typename LF::Raw f0 = fr[0], f1 = fr[1], f2 = fr[2];
            const typename LS::Raw s0 = sr[0], s1 = sr[1], s2 = sr[2];
            c += ngrp;
            const bool more = c < ncol;
            if (more) {
                i += di;
                j += dj;
                if (j >= ny) {
                    j -= ny;
                    i++;
                }
                off = at(i, j);
                fr[0] = LF::raw(u + off);
                fr[1] = LF::raw(v + off);
                fr[2] = LF::raw(w + off);
                sr[0] = LS::raw(su + off);
                sr[1] = LS::raw(sv + off);
                sr[2] = LS::raw(sw + off);
            }
            const D2 f[3] = {LF::run(f0, ok0, ok1, bad), LF::run(f1, ok0, ok1, bad), LF::run(f2, okw0, okw1, bad)};
            const D2 s[3] = {LS::run(s0, ok0, ok1, bad), LS::run(s1, ok0, ok1, bad), LS::run(s2, okw0, okw1, bad)};
#pragma unroll
            for (int q = 0; q < 3; q++) {
                const D2 ps = df_mul(f[q], s[q]);
                acc[4 * q + 0] = df_add(acc[4 * q + 0], ps);
                acc[4 * q + 1] = df_add(acc[4 * q + 1], pw_res_abs(ps));
                acc[4 * q + 2] = df_add(acc[4 * q + 2], s[q]);
                acc[4 * q + 3] = df_add(acc[4 * q + 3], pw_res_abs(s[q]));
            }
            if (!more) break;
        }
    }
    // weighted, in FP64: W(k) times the level-k sums plus W(k+1) times the others
    double vals[PW_RED_STRIDE];
    const double wu0 = ok0 ? wuv[k] : 0.0, wu1 = ok1 ? wuv[k + 1] : 0.0;
    const double ww0 = okw0 ? ww[k] : 0.0, ww1 = okw1 ? ww[k + 1] : 0.0;
#pragma unroll
    for (int q = 0; q < 12; q++) {
        const double w0 = q < 8 ? wu0 : ww0, w1 = q < 8 ? wu1 : ww1;
        vals[q] = w0 * pw_res_join(lx(acc[q].h), lx(acc[q].l)) + w1 * pw_res_join(ly(acc[q].h), ly(acc[q].l));
    }
    vals[12] = bad ? 1.0 : 0.0;
    pw_res_block_tree<PW_RED_FAST_THREADS>(vals, partials + (size_t)blockIdx.x * PW_RED_STRIDE);
    pw_res_finish<PW_RED_FAST_THREADS>(partials);
}

// The plain FP64 pass (used when the fast pass met values outside its range).
template <typename TF, typename TS>
__global__ void __launch_bounds__(PW_RED_THREADS)
pw_residual_exact(const TF *u, const TF *v, const TF *w, const TS *su, const TS *sv, const TS *sw,
                  const double *wuv, const double *ww, int nx, int ny, int nz, int nzp,
                  double *partials) {
    double acc[PW_RED_STRIDE];
#pragma unroll
    for (int q = 0; q < PW_RED_STRIDE; q++) acc[q] = 0.0;
    int64_t n = (int64_t)nx * ny * nz;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        int k = (int)(e % nz);
        int64_t col = e / nz;
        int j = (int)(col % ny), i = (int)(col / ny);
        int64_t off = ((int64_t)(i + 2) * (ny + 4) + (j + 2)) * nzp + k;
        double Wc[3] = {wuv[k], wuv[k], ww[k]};
        double f[3] = {pw_to<double>(u[off]), pw_to<double>(v[off]), pw_to<double>(w[off])};
        double s[3] = {pw_to<double>(su[off]), pw_to<double>(sv[off]), pw_to<double>(sw[off])};
        if (k == nz - 1) {  // lid face: w and sw are 0 by definition
            f[2] = 0.0;
            s[2] = 0.0;
        }
#pragma unroll
        for (int c = 0; c < 3; c++) {
            double ps = f[c] * s[c];
            acc[4 * c + 0] += Wc[c] * ps;
            acc[4 * c + 1] += Wc[c] * fabs(ps);
            acc[4 * c + 2] += Wc[c] * s[c];
            acc[4 * c + 3] += Wc[c] * fabs(s[c]);
        }
    }
    pw_res_block_tree<PW_RED_THREADS>(acc, partials + (size_t)blockIdx.x * PW_RED_STRIDE);
    pw_res_finish<PW_RED_THREADS>(partials);
}

static pw_status pw_residual_launch(bool exact, int nx, int ny, int nz, int nzp, pw_dtype dtype, const double *wuv,
                                    const double *ww, const void *u, const void *v, const void *w,
                                    const void *su, const void *sv, const void *sw, double *scratch,
                                    cudaStream_t st) {
#define PW_RES(TF, TS)                                                                                     \
    do {                                                                                                   \
        if (exact)                                                                                         \
            pw_residual_exact<TF, TS><<<PW_RED_BLOCKS, PW_RED_THREADS, 0, st>>>(                           \
                (const TF *)u, (const TF *)v, (const TF *)w, (const TS *)su, (const TS *)sv,               \
                (const TS *)sw, wuv, ww, nx, ny, nz, nzp, scratch);                                        \
        else                                                                                               \
            pw_residual_fast<TF, TS><<<PW_RED_BLOCKS, PW_RED_FAST_THREADS, 0, st>>>(                       \
                (const TF *)u, (const TF *)v, (const TF *)w, (const TS *)su, (const TS *)sv,               \
                (const TS *)sw, wuv, ww, nx, ny, nz, nzp, scratch);                                        \
    } while (0)
    if (dtype == PW_F64) PW_RES(double, double);
    else if (dtype == PW_F32) PW_RES(float, float);
    else if (dtype == PW_BF16_OUT) PW_RES(__nv_bfloat16, __nv_bfloat16);
    else PW_RES(__nv_bfloat16, float);
#undef PW_RES
    PW_CUDA(cudaGetLastError());
    return PW_OK;
}

pw_status pw_residuals_run(int nx, int ny, int nz, int nzp, pw_dtype dtype, const double *wuv,
                           const double *ww, const void *u, const void *v, const void *w,
                           const void *su, const void *sv, const void *sw, double *scratch,
                           double *staging, double *out, cudaStream_t st) {
    double local[PW_RED_STRIDE];
    double *h = staging ? staging : local;
    for (int pass = 0; pass < 2; pass++) {
        pw_status s = pw_residual_launch(pass == 1, nx, ny, nz, nzp, dtype, wuv, ww, u, v, w, su, sv, sw,
                                         scratch, st);
        if (s != PW_OK) return s;
        PW_CUDA(cudaMemcpyAsync(h, scratch + PW_RED_BLOCKS * PW_RED_STRIDE, PW_RED_STRIDE * sizeof(double),
                                cudaMemcpyDeviceToHost, st));
        PW_CUDA(cudaStreamSynchronize(st));
        // the fast pass stands unless it met values outside its range or a sum
        // of magnitudes is so small that underflow of its terms could matter
        bool redo = h[12] != 0.0;
        for (int q = 1; q < 12; q += 2) redo = redo || (h[q] != 0.0 && fabs(h[q]) < 0x1p-40);
        if (!redo) break;
    }
    for (int q = 0; q < 12; q++) out[q] = h[q];
    return PW_OK;
}

extern "C" pw_status pw_residuals(const pw_mesh *m, const void *u, const void *v, const void *w,
                                  const void *su, const void *sv, const void *sw, double *out,
                                  void *stream) {
    if (!m || !out) return pw_fail(PW_ERR_ARG, "mesh and out must not be NULL");
    pw_status s;
    const void *ps[6] = {u, v, w, su, sv, sw};
    const char *nm[6] = {"u", "v", "w", "su", "sv", "sw"};
    for (int q = 0; q < 6; q++)
        if ((s = pw_check_ptr(ps[q], nm[q])) != PW_OK) return s;
    return pw_residuals_run(m->nx, m->ny, m->nz, m->nzp, m->dtype, m->coef64 + 10 * m->nz, m->coef64 + 11 * m->nz,
                            u, v, w, su, sv, sw, m->partials, m->host_sums, out, (cudaStream_t)stream);
}

extern "C" pw_status pw_residual_ratios(const double *sums, double *out) {
    if (!sums || !out) return pw_fail(PW_ERR_ARG, "sums and out must not be NULL");
    for (int c = 0; c < 3; c++) {
        out[c] = sums[4 * c + 1] != 0.0 ? sums[4 * c] / sums[4 * c + 1] : 0.0;
        out[3 + c] = sums[4 * c + 3] != 0.0 ? sums[4 * c + 2] / sums[4 * c + 3] : 0.0;
    }
    return PW_OK;
}
