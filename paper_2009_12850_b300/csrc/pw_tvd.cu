// pw_tvd.cu -- the positivity-preserving scalar scheme the paper names beside
// PW (section 3.1; section 4 scales PW to its cost): ULTIMATE-limited QUICKEST
// face values in flux form on the C-grid, for cell-centred scalars.
//
//   s = (u(i-1) f_x(i-1) - u(i) f_x(i)) / dx + (v(j-1) f_y(j-1) - v(j) f_y(j)) / dy
//     + fz1(k) w(k-1) f_z(k-1) - fz2(k) w(k) f_z(k)
//   fz1 = rho_w(k-1) / (rho_n dz) = 4 tzc1,  fz2 = rho_w(k) / (rho_n dz) = 4 tzc2
//
// f being the face value of phi: for a face with velocity a between cells L and
// R, the upwind cell C (L when a >= 0, else R), the downwind cell D and the far
// upwind cell U (one beyond C) give, with c = |a| dt / (width of C),
//   q = (phi_C + phi_D)/2 - c (phi_D - phi_C)/2 - (1 - c^2)/6 (phi_D - 2 phi_C + phi_U)
// (QUICKEST, Leonard 1979), held, where phi_C lies strictly between phi_U and
// phi_D, between phi_C and min(phi_D, phi_U + (phi_C - phi_U)/c) (the ULTIMATE
// universal limiter of Leonard 1991, written without the normalised variable);
// elsewhere f = phi_C.  A face whose U cell would lie below the ground or above
// the lid takes phi_C; the ground and lid faces carry nothing.  The
// monotonicity test compares input values only, so it is exact in any
// precision, and both clamps are continuous.
//
// Layout of the work: an x-march over TMA-staged (j,k) planes of u, v, w and
// phi (rows j0-2 .. j0+TJ+1 and a 16-byte k halo: the scheme reaches two cells
// in x, y and z; the mesh's halos are two wide).  A CTA owns TJ rows x 32
// levels, two consecutive levels per thread (the march's per-step work is
// paid once per two values).  Each step takes the newest plane p (column
// i0-2+p) and
//   1. evaluates the y and z face fluxes of that plane: each thread the faces
//      south of and below its two points, row 0's threads also the faces north
//      of the last row, TJ threads of row 1 those above the top level, into one
//      of two shared-memory sets;
//   2. after the step's one CTA barrier (which also frees plane p's ring slot
//      for plane p + NS), forms each point's y + z flux divergence D (held two
//      steps in registers);
//   3. evaluates the x face flux between columns p-3 and p-2 from the thread's
//      own register window phi(p-3 .. p) and writes column p-2's source;
// so each point costs one x face and about 2.2 y/z faces instead of six.
#include <algorithm>
#include <type_traits>

#include "pw_march.cuh"

#define PW_TVD_NS 3   // ring slots (two planes of look-ahead)
#define PW_TVD_KC 32  // levels per CTA (one warp per row)

struct PwTvdGeom {
    int nx, ny, nz, nzp;
    int ti;            // columns marched per CTA
    int nkc;           // k chunks
    long long si, sj;  // strides of the sources (elements)
    double dtdx, dtdy; // dt/dx, dt/dy
    double rdx, rdy;   // 1/dx, 1/dy
    double dt;
    float fdtdx, fdtdy, frdx, frdy, fdt;  // the same rounded to FP32 on the host (FP32 kernels)
};

struct PwTvdSet {
    CUtensorMap phi[PW_MAX_SCALARS];  // box {kb, TJ+4, 1}
    void *out[PW_MAX_SCALARS];
};

// compile-time slot geometry of a storage type: k halo H (16 bytes), box k
// extent KB, elements between the u, v, w, phi planes of a slot (128-byte aligned)
template <typename TS, int TJ>
struct PwTvdShape {
    static constexpr int H = 16 / (int)sizeof(TS);
    static constexpr int KB = PW_TVD_KC + 2 * H;
    static constexpr int PER128 = 128 / (int)sizeof(TS);
    static constexpr int FS = ((TJ + 4) * KB + PER128 - 1) / PER128 * PER128;
};

template <typename TC>
__device__ __forceinline__ TC pw_tvd_div(TC x, TC y) {
    if constexpr (std::is_same<TC, float>::value) return __fdividef(x, y);
    else return x / y;
}

// a * f for the face between cells L and R (phi at L-1, L, R, R+1), velocity a;
// cfp, cfn: dt / width of the upwind cell for a >= 0 (cell L) and a < 0 (cell R);
// farp, farn: the far upwind cell exists for a >= 0 (L-1) and a < 0 (R+1).
// Branch-free: both clamps are formed and the flow decides by selection (the
// quotient is only selected where c |phi_D - phi_U| > |phi_C - phi_U|, so c > 0).
template <typename TC>
__device__ __forceinline__ TC pw_tvd_flux(TC a, TC cfp, TC cfn, TC pl2, TC pl, TC pr, TC pr2, bool farp,
                                          bool farn) {
    const bool pos = a >= TC(0);
    const TC pu = pos ? pl2 : pr2, pc = pos ? pl : pr, pd = pos ? pr : pl;
    const TC c = fabs(a) * (pos ? cfp : cfn);
    const bool up = pu < pc && pc < pd, dn = pd < pc && pc < pu;
    const bool mono = (pos ? farp : farn) && (up || dn);
    const TC q = TC(0.5) * (pc + pd) - TC(0.5) * c * (pd - pc) -
                 (TC(1) - c * c) * (TC(1) / TC(6)) * ((pd - pc) - (pc - pu));
    const TC del = pd - pu, dc = pc - pu;
    // upper end: phi_D, or phi_U + (phi_C - phi_U)/c where that is nearer
    const TC hi = c * fabs(del) > fabs(dc) ? pu + pw_tvd_div(dc, c) : pd;
    const TC f = mono ? (up ? fmax(fmin(q, hi), pc) : fmin(fmax(q, hi), pc)) : pc;
    return a * f;
}

// two consecutive values (levels k, k+1; k even, so the pair is aligned) of a
// staged row, widened to the compute type
template <typename TS, typename TC>
__device__ __forceinline__ void pw_tvd_ld2(const TS *p, TC &a, TC &b) {
    if constexpr (std::is_same<TS, float>::value) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        a = v.x;
        b = v.y;
    } else if constexpr (std::is_same<TS, double>::value) {
        const double2 v = *reinterpret_cast<const double2 *>(p);
        a = (TC)v.x;
        b = (TC)v.y;
    } else {
        const uint32_t v = *reinterpret_cast<const uint32_t *>(p);
        a = __uint_as_float(v << 16);  // bf16 -> f32 is exact
        b = __uint_as_float(v & 0xffff0000u);
    }
}

// the two results of a thread (levels k, k+1; the second only when k+1 < nz)
template <typename TO, typename TC>
__device__ __forceinline__ void pw_tvd_st2(TO *o, TC s0, TC s1, bool two, int beta) {
    if constexpr (std::is_same<TO, __nv_bfloat16>::value) {
        float a = (float)s0, b = (float)s1;
        if (beta) {  // the stored values are read only when accumulating
            a += __bfloat162float(o[0]);
            if (two) b += __bfloat162float(o[1]);
        }
        if (two) *reinterpret_cast<__nv_bfloat162 *>(o) = __floats2bfloat162_rn(a, b);
        else o[0] = __float2bfloat16_rn(a);
    } else {
        using V = typename std::conditional<sizeof(TO) == 8, double2, float2>::type;
        if (two) {
            V v;
            if (beta) {  // the stored values are read only when accumulating
                v = *reinterpret_cast<const V *>(o);
                v.x += (TO)s0;
                v.y += (TO)s1;
            } else {
                v.x = (TO)s0;
                v.y = (TO)s1;
            }
            *reinterpret_cast<V *>(o) = v;
        } else {
            TO a = (TO)s0;
            if (beta) a += o[0];
            o[0] = a;
        }
    }
}

// TJ rows per CTA, TS storage, TC arithmetic, TO source type.  A thread owns
// two levels (k, k+1) of one row; 16 threads cover a row's 32 levels.
//
// Face schedule of a step, per thread (tr, t), k = k0 + 2t:
//   A: the y faces south of its two points (rows j-1 | j),
//   B: the z faces below its two points (levels k-1 | k and k | k+1),
//   C: row 0's threads also take the y faces north of the last row, the
//      first TJ threads of row 1 the z face above the chunk's top level of
//      row r = tid - 16;
// the face above level k is the thread's own second B face; those north of
// its points and above level k+1 are read from shared memory after the
// step's barrier.
template <typename TS, typename TC, typename TO, int TJ>
__global__ void __launch_bounds__(TJ * PW_TVD_KC / 2)
pw_tvd_march(const __grid_constant__ CUtensorMap mu, const __grid_constant__ CUtensorMap mv,
             const __grid_constant__ CUtensorMap mw, const __grid_constant__ PwTvdSet set,
             const double *__restrict__ coef64, const float *__restrict__ coef32, const PwTvdGeom g, int beta,
             int *__restrict__ status) {
    constexpr int KC = PW_TVD_KC, NS = PW_TVD_NS, ROWS = TJ + 4, HK = KC / 2;
    using SH = PwTvdShape<TS, TJ>;
    constexpr int H = SH::H, KB = SH::KB, FS = SH::FS;
    constexpr int NGY = (TJ + 1) * KC, NGZ = TJ * (KC + 1);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if (pw_cta_failed(status)) return;
    const int sc = blockIdx.x / g.nkc, kchunk = blockIdx.x % g.nkc;
    const int j0 = blockIdx.y * TJ, i0 = blockIdx.z * g.ti, k0 = kchunk * KC;
    TS *planes = reinterpret_cast<TS *>(smem_raw);
    TC *Gbuf = reinterpret_cast<TC *>(smem_raw + (size_t)NS * 4 * FS * sizeof(TS));  // two sets of faces
    TC *cft = Gbuf + 2 * (NGY + NGZ);  // dt / dz(K) for K = k0-1 .. k0+KC (0 outside the column)
    uint64_t *bars = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(cft) +
                                                  ((KC + 2) * sizeof(TC) + 15) / 16 * 16);

    const int tid = threadIdx.x, nt = TJ * HK;
    const int tr = tid / HK, t = tid % HK;
    const int j = j0 + tr, k = k0 + 2 * t;
    const bool act0 = j < g.ny && k < g.nz, two = k + 1 < g.nz;
    const int i_end = min(i0 + g.ti, g.nx);
    const int nplanes = i_end - i0 + 4;
    constexpr uint32_t slot_bytes = 4u * ROWS * KB * sizeof(TS);

    if (tid == 0) {
        pw_prefetch_map(&mu);
        pw_prefetch_map(&mv);
        pw_prefetch_map(&mw);
        pw_prefetch_map(&set.phi[sc]);
        for (int s = 0; s < NS; s++) pw_mbar_init(&bars[s], 1);
        pw_fence_barrier_init();
    }
    for (int q = tid; q < KC + 2; q += nt) {
        const int K = k0 - 1 + q;
        // FP32 kernels: one conversion and an FP32 quotient (the FP64 units
        // are slow enough that an FP64 quotient per entry shows in the profile)
        if constexpr (std::is_same<TC, float>::value)
            cft[q] = (K >= 0 && K < g.nz) ? g.fdt / (float)coef64[K] : 0.0f;
        else
            cft[q] = (K >= 0 && K < g.nz) ? (TC)(g.dt / coef64[K]) : TC(0);
    }
    __syncthreads();

    auto slot = [&](int p) { return planes + (size_t)(p % NS) * 4 * FS; };
    auto issue = [&](int p) {
        const int s = p % NS;
        TS *dst = slot(p);
        pw_mbar_expect_tx(&bars[s], slot_bytes);
        const int c0 = k0 - H, c1 = j0, c2 = i0 + p;  // (k0-H, j0-2, i0-2+p) + the halo offset 2
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

    TC cfx, cfy, rdx, rdy;
    if constexpr (std::is_same<TC, float>::value) {
        cfx = g.fdtdx;
        cfy = g.fdtdy;
        rdx = g.frdx;
        rdy = g.frdy;
    } else {
        cfx = g.dtdx;
        cfy = g.dtdy;
        rdx = g.rdx;
        rdy = g.rdy;
    }
    TC fz1[2], fz2[2];
#pragma unroll
    for (int m = 0; m < 2; m++) {
        const int kk = k + m;
        // 4 tzc1, 4 tzc2 (scaling by 4 is exact): the FP32 copies for the FP32 kernels
        if constexpr (std::is_same<TC, float>::value) {
            fz1[m] = (kk > 0 && kk < g.nz) ? 4.0f * coef32[kk] : 0.0f;
            fz2[m] = (kk < g.nz - 1) ? 4.0f * coef32[g.nz + kk] : 0.0f;
        } else {
            fz1[m] = (kk > 0 && kk < g.nz) ? 4.0 * coef64[6 * g.nz + kk] : 0.0;
            fz2[m] = (kk < g.nz - 1) ? 4.0 * coef64[7 * g.nz + kk] : 0.0;
        }
    }
    // B faces: below level k (K = k-1) and below level k+1 (K = k)
    const bool zB0 = k >= 1 && k < g.nz, zB1 = k + 1 < g.nz;
    const TC cfm = cft[2 * t], cf0 = cft[2 * t + 1], cf1 = cft[2 * t + 2];  // dt/dz(k-1), (k), (k+1)
    // C: row 0's threads: the y faces north of row TJ-1 at levels k, k+1;
    // threads HK .. HK+TJ-1: the z face above level k0+KC-1 of row tid-HK
    const int roleC = tid < HK ? 1 : (tid < HK + TJ ? 2 : 0);
    const int rC = tid - HK;
    const int KT = k0 + KC - 1;
    const bool zC = KT < g.nz - 1;
    const TC cfCp = cft[KC], cfCn = cft[KC + 1];
    const bool farCn = KT + 2 < g.nz;

    const int oA = tr * KB + H + 2 * t;            // A: phi rows j-2 .. j+1 at (k, k+1), v(j-1) one row down
    const int oB = (tr + 2) * KB + H + 2 * t - 2;  // B: pairs (k-2, k-1), (k, k+1), (k+2, k+3) of row j
    const int own = (tr + 2) * KB + H + 2 * t;     // this thread's (j, k)
    const int oC = roleC == 1 ? TJ * KB + H + 2 * t : (rC + 2) * KB + H + KC - 2;

    TO *o = reinterpret_cast<TO *>(set.out[sc]) + (long long)(i0 + 2) * g.si + (long long)(j + 2) * g.sj + k;
    TC ph[4][2] = {}, uw[3][2] = {};  // phi at columns c-1 .. c+2, u at c .. c+2 (own points)
    TC D1[2] = {}, D2[2] = {};        // y + z divergence of columns p-1, p-2
    TC Gx_w[2] = {};                  // x flux on the west face of the column written next

    for (int p = 0; p < nplanes; p++) {
        // every thread waits for plane p itself; the step's one CTA barrier
        // (after the face fluxes) shares the outcome
        const bool ok = pw_mbar_wait_bounded(&bars[p % NS], (uint32_t)((p / NS) & 1));
        TC *Gy = Gbuf + (p & 1) * (NGY + NGZ), *Gz = Gy + NGY;
        const TS *P = slot(p);
        const TS *Pu = P, *Pv = P + FS, *Pw = P + 2 * FS, *Pp = P + 3 * FS;
        const bool faces = p >= 2 && p < nplanes - 2;  // columns i0 .. i_end-1
        TC c0v, c1v;  // phi at (k, k+1)
        pw_tvd_ld2<TS, TC>(Pp + own, c0v, c1v);
        TC GA[2] = {}, GB[2] = {};
        if (faces) {
            TC s0, s1, r0, r1, n0, n1, v0, v1;
            pw_tvd_ld2<TS, TC>(Pp + oA, s0, s1);
            pw_tvd_ld2<TS, TC>(Pp + oA + KB, r0, r1);
            pw_tvd_ld2<TS, TC>(Pp + oA + 3 * KB, n0, n1);
            pw_tvd_ld2<TS, TC>(Pv + oA + KB, v0, v1);
            GA[0] = pw_tvd_flux<TC>(v0, cfy, cfy, s0, r0, c0v, n0, true, true);
            GA[1] = pw_tvd_flux<TC>(v1, cfy, cfy, s1, r1, c1v, n1, true, true);
            TC m2, m1, p2, p3, wm, wq, w0, w1;
            pw_tvd_ld2<TS, TC>(Pp + oB, m2, m1);
            pw_tvd_ld2<TS, TC>(Pp + oB + 4, p2, p3);
            pw_tvd_ld2<TS, TC>(Pw + oB, wq, wm);  // w(k-2), w(k-1)
            pw_tvd_ld2<TS, TC>(Pw + oB + 2, w0, w1);
            // every staged value is finite (levels outside the column arrive
            // as 0), so faces below level 0 or past the lid are formed and dropped
            const TC b0 = pw_tvd_flux<TC>(wm, cfm, cf0, m2, m1, c0v, c1v, k >= 2, k + 1 < g.nz);
            const TC b1 = pw_tvd_flux<TC>(w0, cf0, cf1, m1, c0v, c1v, p2, k >= 1, k + 2 < g.nz);
            GB[0] = zB0 ? b0 : TC(0);
            GB[1] = zB1 ? b1 : TC(0);
            (void)wq;
            (void)w1;
            (void)p3;
            if (roleC == 1) {
                TC a0, a1, e0, e1, f0, f1, h0, h1, q0, q1;
                pw_tvd_ld2<TS, TC>(Pp + oC, a0, a1);
                pw_tvd_ld2<TS, TC>(Pp + oC + KB, e0, e1);
                pw_tvd_ld2<TS, TC>(Pp + oC + 2 * KB, f0, f1);
                pw_tvd_ld2<TS, TC>(Pp + oC + 3 * KB, h0, h1);
                pw_tvd_ld2<TS, TC>(Pv + oC + KB, q0, q1);
                Gy[TJ * KC + 2 * t] = pw_tvd_flux<TC>(q0, cfy, cfy, a0, e0, f0, h0, true, true);
                Gy[TJ * KC + 2 * t + 1] = pw_tvd_flux<TC>(q1, cfy, cfy, a1, e1, f1, h1, true, true);
            } else if (roleC == 2) {
                TC a0, a1, e0, e1, q0, q1;  // levels KT-1 .. KT+2 and w(KT)
                pw_tvd_ld2<TS, TC>(Pp + oC, a0, a1);
                pw_tvd_ld2<TS, TC>(Pp + oC + 2, e0, e1);
                pw_tvd_ld2<TS, TC>(Pw + oC, q0, q1);
                Gz[rC * (KC + 1) + KC] = zC ? pw_tvd_flux<TC>(q1, cfCp, cfCn, a0, a1, e0, e1, true, farCn) : TC(0);
            }
            Gy[tr * KC + 2 * t] = GA[0];
            Gy[tr * KC + 2 * t + 1] = GA[1];
            Gz[tr * (KC + 1) + 2 * t] = GB[0];
            Gz[tr * (KC + 1) + 2 * t + 1] = GB[1];
        }
        // own values of the newest plane
#pragma unroll
        for (int m = 0; m < 2; m++) {
            ph[0][m] = ph[1][m];
            ph[1][m] = ph[2][m];
            ph[2][m] = ph[3][m];
            uw[0][m] = uw[1][m];
            uw[1][m] = uw[2][m];
        }
        ph[3][0] = c0v;
        ph[3][1] = c1v;
        pw_tvd_ld2<TS, TC>(Pu + own, uw[2][0], uw[2][1]);
        if (!__syncthreads_and(ok)) {
            give_up(p);
            return;
        }
        // every thread is done reading plane p (faces and its own values): its
        // slot takes plane p + NS
        if (tid == 0 && p + NS < nplanes) {
            issue(p + NS);
            issued = p + NS + 1;
        }
        TC D[2] = {};
        if (faces) {
            D[0] = (GA[0] - Gy[(tr + 1) * KC + 2 * t]) * rdy + fz1[0] * GB[0] - fz2[0] * GB[1];
            D[1] = (GA[1] - Gy[(tr + 1) * KC + 2 * t + 1]) * rdy + fz1[1] * GB[1] -
                   fz2[1] * Gz[tr * (KC + 1) + 2 * t + 2];
        }
        if (p >= 3) {
            // x faces between columns c = i0+p-4 and c+1: phi(c-1 .. c+2), u(c)
            TC Gx[2];
#pragma unroll
            for (int m = 0; m < 2; m++)
                Gx[m] = pw_tvd_flux<TC>(uw[0][m], cfx, cfx, ph[0][m], ph[1][m], ph[2][m], ph[3][m], true, true);
            if (p >= 4) {
                if (act0) pw_tvd_st2<TO, TC>(o, (Gx_w[0] - Gx[0]) * rdx + D2[0], (Gx_w[1] - Gx[1]) * rdx + D2[1],
                                             two, beta);
                o += g.si;
            }
            Gx_w[0] = Gx[0];
            Gx_w[1] = Gx[1];
        }
#pragma unroll
        for (int m = 0; m < 2; m++) {
            D2[m] = D1[m];
            D1[m] = D[m];
        }
    }
    __syncthreads();
    if (tid == 0)
        for (int s = 0; s < NS; s++) pw_mbar_inval(&bars[s]);
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
template <typename TS, typename TC, typename TO, int TJ>
static pw_status pw_launch_tvd_t(const pw_mesh *m, const void *u, const void *v, const void *w, int n,
                                 const void *const *phi, void *const *sphi, double dt, int beta,
                                 cudaStream_t st, int tile_i) {
    constexpr int KC = PW_TVD_KC, NS = PW_TVD_NS;
    PwTvdGeom g;
    using SH = PwTvdShape<TS, TJ>;
    g.nx = m->nx;
    g.ny = m->ny;
    g.nz = m->nz;
    g.nzp = m->nzp;
    g.nkc = (m->nz + KC - 1) / KC;
    const long tiles = (long)((m->ny + TJ - 1) / TJ) * g.nkc * n;
    g.si = m->si;
    g.sj = m->sj;
    g.dtdx = dt / m->dx;
    g.dtdy = dt / m->dy;
    g.rdx = 1.0 / m->dx;
    g.rdy = 1.0 / m->dy;
    g.dt = dt;
    g.fdtdx = (float)g.dtdx;
    g.fdtdy = (float)g.dtdy;
    g.frdx = (float)g.rdx;
    g.frdy = (float)g.rdy;
    g.fdt = (float)dt;
    const size_t smem = (size_t)NS * 4 * SH::FS * sizeof(TS) +
                        (size_t)2 * ((TJ + 1) * KC + TJ * (KC + 1)) * sizeof(TC) +
                        ((KC + 2) * sizeof(TC) + 15) / 16 * 16 + NS * sizeof(uint64_t);
    if (smem > 226 * 1024) return pw_fail(PW_ERR_SHAPE, "tvd: %zu bytes of shared memory", smem);
    CUtensorMap maps[3];
    const void *f[3] = {u, v, w};
    for (int q = 0; q < 3; q++) {
        pw_status s = pw_make_field_map(&maps[q], f[q], m->dtype, m->nx, m->ny, m->nzp, pw_kdim(m->nz, q), SH::KB,
                                        TJ + 4);
        if (s != PW_OK) return s;
    }
    PwTvdSet set;
    memset(&set, 0, sizeof(set));
    for (int q = 0; q < n; q++) {
        pw_status s = pw_make_field_map(&set.phi[q], phi[q], m->dtype, m->nx, m->ny, m->nzp, m->nz, SH::KB, TJ + 4);
        if (s != PW_OK) return s;
        set.out[q] = sphi[q];
    }
    auto kern = pw_tvd_march<TS, TC, TO, TJ>;
    PW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // a CTA marches ti columns from ti + 4 planes
    g.ti = pw_pick_tile_i(m, tile_i, tiles, pw_slots(m, kern, TJ * KC / 2, smem), 4);
    // the scalar and the k chunk are the fastest grid indices: the CTAs of one
    // tile run together and share the wind and the k-halo levels through L2
    dim3 grid((unsigned)(g.nkc * n), (unsigned)((m->ny + TJ - 1) / TJ), (unsigned)((m->nx + g.ti - 1) / g.ti));
    if (grid.y > 65535 || grid.z > 65535) return pw_fail(PW_ERR_SHAPE, "tvd: grid too large");
    kern<<<grid, TJ * KC / 2, smem, st>>>(maps[0], maps[1], maps[2], set, m->coef64, m->coef32, g, beta,
                                          m->status);
    PW_CUDA(cudaGetLastError());
    return PW_OK;
}

static pw_status pw_launch_tvd(const pw_mesh *m, const void *u, const void *v, const void *w, int n,
                               const void *const *phi, void *const *sphi, double dt, int beta, cudaStream_t st) {
    const int ti = m->tile_i;
    switch (m->dtype) {
        case PW_F64:
            if (m->algo == PW_ALGO_F64_SPLIT) return pw_launch_tvd_split(m, u, v, w, n, phi, sphi, dt, beta, st);
            return pw_launch_tvd_t<double, double, double, 8>(m, u, v, w, n, phi, sphi, dt, beta, st, ti);
        case PW_F32:
            return pw_launch_tvd_t<float, float, float, 8>(m, u, v, w, n, phi, sphi, dt, beta, st, ti);
        case PW_BF16:
            return pw_launch_tvd_t<__nv_bfloat16, float, float, 8>(m, u, v, w, n, phi, sphi, dt, beta, st, ti);
        case PW_BF16_OUT:
            return pw_launch_tvd_t<__nv_bfloat16, float, __nv_bfloat16, 8>(m, u, v, w, n, phi, sphi, dt, beta, st,
                                                                           ti);
    }
    return pw_fail(PW_ERR_DTYPE, "unknown dtype");
}

extern "C" pw_status pw_advect_tvd(const pw_mesh *m, const void *u, const void *v, const void *w, int n,
                                   const void *const *phi, void *const *sphi, double dt, int beta, void *stream) {
    if (!m) return pw_fail(PW_ERR_ARG, "mesh is NULL");
    if (beta != 0 && beta != 1) return pw_fail(PW_ERR_ARG, "beta must be 0 or 1");
    if (!(dt > 0.0) || dt - dt != 0.0) return pw_fail(PW_ERR_ARG, "dt must be finite and positive");
    if (n < 1 || n > PW_MAX_SCALARS) return pw_fail(PW_ERR_ARG, "n = %d scalars (1..%d)", n, PW_MAX_SCALARS);
    if (!phi || !sphi) return pw_fail(PW_ERR_ARG, "scalar pointer arrays are NULL");
    const void *wind[3] = {u, v, w};
    const char *wn[3] = {"u", "v", "w"};
    for (int q = 0; q < 3; q++) {
        pw_status s = pw_check_ptr(wind[q], wn[q]);
        if (s != PW_OK) return s;
    }
    for (int a = 0; a < n; a++) {
        pw_status s = pw_check_ptr(phi[a], "phi[a]");
        if (s != PW_OK) return s;
        s = pw_check_ptr(sphi[a], "sphi[a]");
        if (s != PW_OK) return s;
        for (int q = 0; q < 3; q++)
            if (sphi[a] == wind[q]) return pw_fail(PW_ERR_ARG, "output %d aliases %s", a, wn[q]);
        for (int b = 0; b < n; b++) {
            if (sphi[a] == phi[b]) return pw_fail(PW_ERR_ARG, "output %d aliases phi[%d]", a, b);
            if (b > a && sphi[a] == sphi[b]) return pw_fail(PW_ERR_ARG, "outputs %d and %d alias", a, b);
        }
    }
    return pw_launch_tvd(m, u, v, w, n, phi, sphi, dt, beta, (cudaStream_t)stream);
}
