// pw_tvd_split.cu -- the ULTIMATE-QUICKEST scalar scheme (section 3.1's
// positivity-preserving scheme; the operator is the one of pw_tvd.cu) for FP64
// meshes, in double-float arithmetic on the FP32 pipe (the default for FP64,
// PW_ALGO_F64_SPLIT): B300's FP64 units run at ~1/70 of the FP32 rate, and a
// face costs ~35 FP64 operations natively.
//
// What stays exact.  Every decision of the scheme is taken on exact values,
// as in the FP64 definition: the flow direction from the sign of a, the
// monotonicity test from the signs of the FP64 differences phi_C - phi_U and
// phi_D - phi_C (IEEE differences are 0 only for equal operands and carry the
// true sign), both read from the sign and magnitude bits.  The two differences
// are the only FP64 arithmetic of a face.
//
// The rest is double-float (a value carried as an unevaluated float pair
// h + l, ~47 significant bits, the products by FMA-exact transforms): the
// wind, phi_C and the two differences are split with integer bit operations
// (scaled by 2^8, so the fluxes and the source come out scaled by 2^16 and the
// final join removes it); then, relative to phi_C with d0 = phi_C - phi_U and
// d1 = phi_D - phi_C,
//   c = |a| cf,  q - phi_C = (1 - c) (d1/2 - (1 + c)/6 (d1 - d0)),
//   B = d1 if c |d1| < |d0| max(1 - c, 0), else d0 max(1 - c, 0) / c,
//   f = phi_C + (q - phi_C) held between 0 and B,  flux = a f,
// the limiter's window [phi_C, min(phi_D, phi_U + d0/c)] written relative to
// phi_C (B is the end nearer 0; it closes for c >= 1).  The quotient is the
// FP32 quotient corrected once by its double-float remainder (Dekker 1971).
// A face's rounding error is a few units of 2^-46 of |a| (|phi_U| + |phi_C| +
// |phi_D|), far inside the FP64 tolerance of 1e-12 of the condition sum.
//
// Range (as for the PW split kernels): winds below 2^40 and scalars below 2^60
// in magnitude; larger values, NaN and Inf read as 0 and set PW_ERR_RANGE in
// the mesh status word.
//
// The work layout is pw_tvd.cu's x-march (8 rows x 32 levels per CTA, one
// level per thread, the y and z faces of each plane shared through shared
// memory, the x face carried along the march), over raw FP64 planes.
#include <algorithm>

#include "pw_df.cuh"
#include "pw_internal.h"

#define PW_TVDS_NS 4   // ring slots (three planes of look-ahead)
#define PW_TVDS_KC 32  // levels per CTA (one warp per row)

struct PwTvdSplitGeom {
    int nx, ny, nz;
    int ti;            // columns marched per CTA
    int nkc;           // k chunks
    long long si, sj;  // strides of the sources (elements)
    double dtdx, dtdy, rdx, rdy, dt;
};

struct PwTvdSplitSet {
    CUtensorMap phi[PW_MAX_SCALARS];  // box {36, TJ+4, 1} of doubles
    double *out[PW_MAX_SCALARS];
};

// ---------------------------------------------------------------------------
// scalar double-float values (the packed pairs of pw_df.cuh hold two levels;
// a face here is one value)
// ---------------------------------------------------------------------------
struct DF {
    float h, l;
};
__device__ __forceinline__ DF dfs_neg(DF a) { return DF{-a.h, -a.l}; }
// lazy sum: TwoSum of the high parts, low parts added
__device__ __forceinline__ DF dfs_add(DF a, DF b) {
    const float s = a.h + b.h, bb = s - a.h;
    const float e = (a.h - (s - bb)) + (b.h - bb);
    return DF{s, e + (a.l + b.l)};
}
__device__ __forceinline__ DF dfs_sub(DF a, DF b) { return dfs_add(a, dfs_neg(b)); }
// lazy product (the l*l term, below 2^-46 of the product, is dropped)
__device__ __forceinline__ DF dfs_mul(DF a, DF b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return DF{p, e};
}
// the value rounded to float: its sign is the sign of h + l exactly
__device__ __forceinline__ float dfs_val(DF a) { return a.h + a.l; }
// n / d for d > 0: the FP32 quotient q0 and one correction by the remainder
// n - q0 d (its leading part exact by FMA); relative error ~2^-44
__device__ __forceinline__ DF dfs_div(DF n, DF d) {
    const float r = __fdividef(1.0f, d.h);
    const float q0 = n.h * r;
    float rem = fmaf(-q0, d.h, n.h);
    rem = rem + n.l;
    rem = fmaf(-q0, d.l, rem);
    return DF{q0, rem * r};
}
__device__ __forceinline__ DF dfs_sel(bool c, DF a, DF b) { return DF{c ? a.h : b.h, c ? a.l : b.l}; }

// sign of a double from its bits: -1, 0 or +1 (-0 counts as 0).  The words
// are taken through an opaque move so that the test stays on the integer
// units: written as a comparison of the double, it runs on the FP64 pipe,
// which then bounds the whole kernel.
__device__ __forceinline__ int pw_dsign(double x) {
    uint32_t lo, hi;
    asm volatile("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(x));
    return ((hi << 1) | lo) == 0u ? 0 : ((int)hi < 0 ? -1 : 1);
}

// a double split into a 2^8-scaled double-float (range flag into `bad`)
__device__ __forceinline__ DF pw_dsplit(double x, uint32_t ehi, bool &bad) {
    DF r;
    split_words((uint32_t)__double2loint(x), (uint32_t)__double2hiint(x), r.h, r.l, ehi, bad);
    return r;
}

// a * f (scaled 2^16) for the face between cells L and R (phi at L-1, L, R,
// R+1), velocity a; cfp, cfn: dt / width of the upwind cell for a >= 0 (cell
// L) and a < 0 (cell R), times 2^-8; farp, farn: the far upwind cell exists
// for a >= 0 (L-1) and a < 0 (R+1)
__device__ __forceinline__ DF pw_tvds_flux(double a, DF cfp, DF cfn, double pl2, double pl, double pr, double pr2,
                                           bool farp, bool farn, bool &bad) {
    const bool pos = pw_dsign(a) >= 0;
    const double pu = pos ? pl2 : pr2, pc = pos ? pl : pr, pd = pos ? pr : pl;
    const double d0 = pc - pu, d1 = pd - pc;  // the FP64 arithmetic of the face
    const int s0 = pw_dsign(d0), s1 = pw_dsign(d1);
    const bool mono = (pos ? farp : farn) && s0 != 0 && s0 == s1;
    const DF A = pw_dsplit(a, PW_SPLIT_WIND_EHI, bad);
    const DF P = pw_dsplit(pc, PW_SPLIT_SCALAR_EHI, bad);
    const DF D0 = pw_dsplit(d0, PW_SPLIT_SCALAR_EHI, bad);
    const DF D1 = pw_dsplit(d1, PW_SPLIT_SCALAR_EHI, bad);
    // the two parts of a split value carry its sign, so |x| is |h| + |l|
    const DF c = dfs_mul(DF{fabsf(A.h), fabsf(A.l)}, pos ? cfp : cfn);  // unscaled
    constexpr float six_h = (float)(1.0 / 6.0), six_l = (float)(1.0 / 6.0 - (double)six_h);
    const DF one{1.0f, 0.0f}, sixth{six_h, six_l};  // 1/6 as h + l (folded by the compiler)
    const DF w1 = dfs_sub(one, c);
    const DF k6 = dfs_add(dfs_mul(c, sixth), sixth);  // (1 + c) / 6
    const DF inner = dfs_sub(DF{0.5f * D1.h, 0.5f * D1.l}, dfs_mul(k6, dfs_sub(D1, D0)));
    const DF tq = dfs_mul(w1, inner);  // q - phi_C
    const DF w = dfs_val(w1) > 0.0f ? w1 : DF{0.0f, 0.0f};
    const DF aD1{fabsf(D1.h), fabsf(D1.l)}, aD0{fabsf(D0.h), fabsf(D0.l)};
    const bool nearD = dfs_val(dfs_sub(dfs_mul(c, aD1), dfs_mul(aD0, w))) < 0.0f;
    // the window's end nearer 0 (the quotient is only taken when c > 0)
    const DF B = nearD ? D1 : dfs_div(dfs_mul(D0, w), c);
    const float sB = dfs_val(B), sq = dfs_val(tq), sd = dfs_val(dfs_sub(tq, B));
    const bool beyond = sB >= 0.0f ? sd > 0.0f : sd < 0.0f;  // tq past B
    const bool behind = sB >= 0.0f ? sq < 0.0f : sq > 0.0f;  // tq on the far side of 0
    const DF t = behind ? DF{0.0f, 0.0f} : (beyond ? B : tq);
    const DF F = mono ? dfs_add(P, t) : P;
    return dfs_mul(A, F);
}

// shared-memory table of a CTA: per level K = k0-1 .. k0+KC of the chunk,
// dt / dz(K) times 2^-8 (the Courant factor of a z face whose upwind cell is
// K); per level k0 .. k0+KC-1, fz1 and fz2; then dt/dx and dt/dy (times 2^-8)
// and 1/dx, 1/dy, all as double-float pairs split from FP64
#define PW_TVDS_CTAB (3 * PW_TVDS_KC + 2 + 4)

// split of an FP64 coefficient into (hi, lo) floats (FP64 operations: done
// once per CTA for the table)
__device__ __forceinline__ DF pw_cpair(double c) {
    const float h = (float)c;
    return DF{h, (float)(c - (double)h)};
}

template <int TJ>
__global__ void __launch_bounds__(TJ * PW_TVDS_KC)
pw_tvd_split_march(const __grid_constant__ CUtensorMap mu, const __grid_constant__ CUtensorMap mv,
                   const __grid_constant__ CUtensorMap mw, const __grid_constant__ PwTvdSplitSet set,
                   const double *__restrict__ coef64, const PwTvdSplitGeom g, int beta, int *__restrict__ status) {
    constexpr int KC = PW_TVDS_KC, NS = PW_TVDS_NS, ROWS = TJ + 4;
    constexpr int H = 2, KB = KC + 2 * H, FS = ((ROWS * KB + 15) / 16) * 16;  // doubles
    constexpr int NGY = (TJ + 1) * KC, NGZ = TJ * (KC + 1);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if (pw_cta_failed(status)) return;
    const int sc = blockIdx.x / g.nkc, kchunk = blockIdx.x % g.nkc;
    const int j0 = blockIdx.y * TJ, i0 = blockIdx.z * g.ti, k0 = kchunk * KC;
    double *planes = reinterpret_cast<double *>(smem_raw);
    DF *Gbuf = reinterpret_cast<DF *>(smem_raw + (size_t)NS * 4 * FS * sizeof(double));  // two sets of faces
    DF *ctab = Gbuf + 2 * (NGY + NGZ);
    uint64_t *bars = reinterpret_cast<uint64_t *>(ctab + PW_TVDS_CTAB);

    const int tid = threadIdx.x, nt = TJ * KC;
    const int tr = tid / KC, tl = tid % KC;
    const int j = j0 + tr, k = k0 + tl;
    const bool active = j < g.ny && k < g.nz;
    const int i_end = min(i0 + g.ti, g.nx);
    const int nplanes = i_end - i0 + 4;
    constexpr uint32_t slot_bytes = 4u * ROWS * KB * sizeof(double);

    if (tid == 0) {
        pw_prefetch_map(&mu);
        pw_prefetch_map(&mv);
        pw_prefetch_map(&mw);
        pw_prefetch_map(&set.phi[sc]);
        for (int s = 0; s < NS; s++) pw_mbar_init(&bars[s], 1);
        pw_fence_barrier_init();
    }
    for (int t = tid; t < PW_TVDS_CTAB; t += nt) {
        double c = 0.0;
        if (t < KC + 2) {
            const int K = k0 - 1 + t;
            if (K >= 0 && K < g.nz) c = g.dt / coef64[K] * 0x1p-8;
        } else if (t < 2 * KC + 2) {
            const int kk = k0 + t - (KC + 2);
            if (kk > 0 && kk < g.nz) c = 4.0 * coef64[6 * g.nz + kk];
        } else if (t < 3 * KC + 2) {
            const int kk = k0 + t - (2 * KC + 2);
            if (kk < g.nz - 1) c = 4.0 * coef64[7 * g.nz + kk];
        } else {
            const int q = t - (3 * KC + 2);
            c = q == 0 ? g.dtdx * 0x1p-8 : q == 1 ? g.dtdy * 0x1p-8 : q == 2 ? g.rdx : g.rdy;
        }
        ctab[t] = pw_cpair(c);
    }
    __syncthreads();

    auto slot = [&](int p) { return planes + (size_t)(p % NS) * 4 * FS; };
    auto issue = [&](int p) {
        const int s = p % NS;
        double *dst = slot(p);
        pw_mbar_expect_tx(&bars[s], slot_bytes);
        const int c0 = k0 - H, c1 = j0, c2 = i0 + p;  // (k0-2, j0-2, i0-2+p) + the halo offset 2
        pw_tma_load_3d(dst, &mu, c0, c1, c2, &bars[s]);
        pw_tma_load_3d(dst + FS, &mv, c0, c1, c2, &bars[s]);
        pw_tma_load_3d(dst + 2 * FS, &mw, c0, c1, c2, &bars[s]);
        pw_tma_load_3d(dst + 3 * FS, &set.phi[sc], c0, c1, c2, &bars[s]);
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

    const DF cfx = ctab[3 * KC + 2], cfy = ctab[3 * KC + 3], rdx = ctab[3 * KC + 4], rdy = ctab[3 * KC + 5];
    const DF fz1 = ctab[KC + 2 + tl], fz2 = ctab[2 * KC + 2 + tl];
    // B: the face below level k (K = k-1): exists for 1 <= k <= nz-1
    const bool zB = k >= 1 && k < g.nz;
    const DF cfBp = ctab[tl], cfBn = ctab[tl + 1];
    const bool farBp = k >= 2, farBn = k + 1 < g.nz;
    // C: warp 0: the y face north of row TJ-1; warp 1, lane r < TJ: the z face
    // above level k0+KC-1 of row r
    const int roleC = tid < KC ? 1 : (tid < KC + TJ ? 2 : 0);
    const int rC = tid - KC;
    const int KT = k0 + KC - 1;
    const bool zC = KT < g.nz - 1;
    const DF cfCp = ctab[KC], cfCn = ctab[KC + 1];
    const bool farCn = KT + 2 < g.nz;

    const int oA = tr * KB + H + tl;            // A: phi rows j-2 .. j+1, v(j-1) one row down
    const int oB = (tr + 2) * KB + H + tl - 2;  // B: levels k-2 .. k+1 of row j; w(k-1)
    const int own = (tr + 2) * KB + H + tl;     // this thread's (j, k)
    const int oC = roleC == 1 ? TJ * KB + H + tl : (rC + 2) * KB + H + KC - 2;

    double *o = set.out[sc] + (long long)(i0 + 2) * g.si + (long long)(j + 2) * g.sj + k;
    bool bad = false;
    double ph[4] = {0.0, 0.0, 0.0, 0.0};  // phi at columns c-1 .. c+2 (own point)
    double uw[3] = {0.0, 0.0, 0.0};       // u at columns c .. c+2
    const DF zero{0.0f, 0.0f};
    DF D1 = zero, D2 = zero;  // y + z divergence of columns p-1, p-2 (scaled 2^16)
    DF Gx_w = zero;           // x flux on the west face of the column written next

    for (int p = 0; p < nplanes; p++) {
        const bool ok = pw_mbar_wait_bounded(&bars[p % NS], (uint32_t)((p / NS) & 1));
        DF *Gy = Gbuf + (p & 1) * (NGY + NGZ), *Gz = Gy + NGY;
        const double *P = slot(p);
        const double *Pu = P, *Pv = P + FS, *Pw = P + 2 * FS, *Pp = P + 3 * FS;
        const bool faces = p >= 2 && p < nplanes - 2;  // columns i0 .. i_end-1
        const double pC = Pp[own];
        DF GA = zero, GB = zero;
        if (faces) {
            GA = pw_tvds_flux(Pv[oA + KB], cfy, cfy, Pp[oA], Pp[oA + KB], pC, Pp[oA + 3 * KB], true, true, bad);
            // every staged value is finite (levels outside the column arrive as
            // 0), so the face below level 0 or past the lid is formed and dropped
            GB = pw_tvds_flux(Pw[oB + 1], cfBp, cfBn, Pp[oB], Pp[oB + 1], pC, Pp[oB + 3], farBp, farBn, bad);
            GB = zB ? GB : zero;
            if (roleC == 1) {
                Gy[TJ * KC + tl] = pw_tvds_flux(Pv[oC + KB], cfy, cfy, Pp[oC], Pp[oC + KB], Pp[oC + 2 * KB],
                                                Pp[oC + 3 * KB], true, true, bad);
            } else if (roleC == 2) {
                const DF G = pw_tvds_flux(Pw[oC + 1], cfCp, cfCn, Pp[oC], Pp[oC + 1], Pp[oC + 2], Pp[oC + 3], true,
                                          farCn, bad);
                Gz[rC * (KC + 1) + KC] = zC ? G : zero;
            }
            Gy[tr * KC + tl] = GA;
            Gz[tr * (KC + 1) + tl] = GB;
        }
        ph[0] = ph[1];
        ph[1] = ph[2];
        ph[2] = ph[3];
        ph[3] = pC;
        uw[0] = uw[1];
        uw[1] = uw[2];
        uw[2] = Pu[own];
        if (!__syncthreads_and(ok)) {
            give_up(p);
            return;
        }
        // every thread is done reading plane p: its slot takes plane p + NS
        if (tid == 0 && p + NS < nplanes) {
            issue(p + NS);
            issued = p + NS + 1;
        }
        DF D = zero;
        if (faces)
            D = dfs_add(dfs_mul(dfs_sub(GA, Gy[(tr + 1) * KC + tl]), rdy),
                        dfs_sub(dfs_mul(fz1, GB), dfs_mul(fz2, Gz[tr * (KC + 1) + tl + 1])));
        if (p >= 3) {
            // x face between columns c = i0+p-4 and c+1: phi(c-1 .. c+2), u(c)
            const DF Gx = pw_tvds_flux(uw[0], cfx, cfx, ph[0], ph[1], ph[2], ph[3], true, true, bad);
            if (p >= 4 && active) {
                const DF s = dfs_add(dfs_mul(dfs_sub(Gx_w, Gx), rdx), D2);
                double r = join(s.h, s.l);
                if (beta) r += *o;  // the stored value is read only when accumulating
                *o = r;
            }
            if (p >= 4) o += g.si;
            Gx_w = Gx;
        }
        D2 = D1;
        D1 = D;
    }
    // every thread reaches this point (inactive points only skip the stores)
    if (__syncthreads_or(bad) && tid == 0) atomicOr(status + PW_STATUS_RANGE_WORD, 1);
    if (tid == 0)
        for (int s = 0; s < NS; s++) pw_mbar_inval(&bars[s]);
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
pw_status pw_launch_tvd_split(const pw_mesh *m, const void *u, const void *v, const void *w, int n,
                              const void *const *phi, void *const *sphi, double dt, int beta, cudaStream_t st) {
    constexpr int TJ = 8, KC = PW_TVDS_KC, NS = PW_TVDS_NS, KB = KC + 4;
    constexpr int FS = (((TJ + 4) * KB + 15) / 16) * 16;
    PwTvdSplitGeom g;
    g.nx = m->nx;
    g.ny = m->ny;
    g.nz = m->nz;
    g.nkc = (m->nz + KC - 1) / KC;
    g.si = m->si;
    g.sj = m->sj;
    g.dtdx = dt / m->dx;
    g.dtdy = dt / m->dy;
    g.rdx = 1.0 / m->dx;
    g.rdy = 1.0 / m->dy;
    g.dt = dt;
    const size_t smem = (size_t)NS * 4 * FS * sizeof(double) +
                        (size_t)2 * ((TJ + 1) * KC + TJ * (KC + 1)) * sizeof(DF) + PW_TVDS_CTAB * sizeof(DF) +
                        NS * sizeof(uint64_t);
    if (smem > 226 * 1024) return pw_fail(PW_ERR_SHAPE, "tvd split: %zu bytes of shared memory", smem);
    CUtensorMap maps[3];
    const void *f[3] = {u, v, w};
    for (int q = 0; q < 3; q++) {
        pw_status s = pw_make_field_map(&maps[q], f[q], PW_F64, m->nx, m->ny, m->nzp, pw_kdim(m->nz, q), KB, TJ + 4);
        if (s != PW_OK) return s;
    }
    PwTvdSplitSet set;
    memset(&set, 0, sizeof(set));
    for (int q = 0; q < n; q++) {
        pw_status s = pw_make_field_map(&set.phi[q], phi[q], PW_F64, m->nx, m->ny, m->nzp, m->nz, KB, TJ + 4);
        if (s != PW_OK) return s;
        set.out[q] = (double *)sphi[q];
    }
    auto kern = pw_tvd_split_march<TJ>;
    PW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long tiles = (long)((m->ny + TJ - 1) / TJ) * g.nkc * n;
    // a CTA marches ti columns from ti + 4 planes
    g.ti = pw_pick_tile_i(m, m->tile_i, tiles, pw_slots(m, kern, TJ * KC, smem), 4);
    // the scalar and the k chunk are the fastest grid indices (the CTAs of a
    // tile share the wind and the k-halo levels through L2)
    dim3 grid((unsigned)(g.nkc * n), (unsigned)((m->ny + TJ - 1) / TJ), (unsigned)((m->nx + g.ti - 1) / g.ti));
    if (grid.y > 65535 || grid.z > 65535) return pw_fail(PW_ERR_SHAPE, "tvd split: grid too large");
    kern<<<grid, TJ * KC, smem, st>>>(maps[0], maps[1], maps[2], set, m->coef64, g, beta, m->status);
    PW_CUDA(cudaGetLastError());
    return PW_OK;
}
