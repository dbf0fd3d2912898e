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
// levels, one level per thread.  Each step takes the newest plane p (column
// i0-2+p) and
//   1. evaluates the y and z face fluxes of that plane: each thread the faces
//      south of and below its point, warps 0 and 1 also the faces north of the
//      last row and above the top level, into one of two shared-memory sets;
//   2. after the step's one CTA barrier (which also frees plane p's ring slot
//      for plane p + NS), forms each point's y + z flux divergence D (held two
//      steps in registers);
//   3. evaluates the x face flux between columns p-3 and p-2 from the thread's
//      own register window phi(p-3 .. p) and writes column p-2's source;
// so each point costs one x face and about 2.2 y/z faces instead of six.
#include <algorithm>
#include <type_traits>

#include "pw_march.cuh"

#define PW_TVD_NS 4   // ring slots (three planes of look-ahead)
#define PW_TVD_KC 32  // levels per CTA (one warp per row)

struct PwTvdGeom {
    int nx, ny, nz, nzp;
    int ti;            // columns marched per CTA
    int nkc;           // k chunks
    long long si, sj;  // strides of the sources (elements)
    double dtdx, dtdy; // dt/dx, dt/dy
    double rdx, rdy;   // 1/dx, 1/dy
    double dt;
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

// TJ rows per CTA, TS storage, TC arithmetic, TO source type.
//
// Face schedule of a step, per thread (tr, tl) = (row, level in the chunk):
//   A: the y face south of its point (rows j-1 | j),
//   B: the z face below its point (levels k-1 | k),
//   C: warp 0 takes the y faces north of the last row, lanes 0..TJ-1 of warp 1
//      the z faces above the chunk's top level;
// a thread keeps its own A and B fluxes and reads the north and upper ones
// from shared memory after the step's barrier.
template <typename TS, typename TC, typename TO, int TJ>
__global__ void __launch_bounds__(TJ * PW_TVD_KC)
pw_tvd_march(const __grid_constant__ CUtensorMap mu, const __grid_constant__ CUtensorMap mv,
             const __grid_constant__ CUtensorMap mw, const __grid_constant__ PwTvdSet set,
             const double *__restrict__ coef64, const PwTvdGeom g, int beta, int *__restrict__ status) {
    constexpr int KC = PW_TVD_KC, NS = PW_TVD_NS, ROWS = TJ + 4;
    using SH = PwTvdShape<TS, TJ>;
    constexpr int H = SH::H, KB = SH::KB, FS = SH::FS;
    constexpr int NGY = (TJ + 1) * KC, NGZ = TJ * (KC + 1);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if (pw_cta_failed(status)) return;
    const int sc = blockIdx.x / g.nkc, kchunk = blockIdx.x % g.nkc;
    const int j0 = blockIdx.y * TJ, i0 = blockIdx.z * g.ti, k0 = kchunk * KC;
    TS *planes = reinterpret_cast<TS *>(smem_raw);
    TC *Gbuf = reinterpret_cast<TC *>(smem_raw + (size_t)NS * 4 * FS * sizeof(TS));  // two sets of faces
    uint64_t *bars = reinterpret_cast<uint64_t *>(Gbuf + 2 * (NGY + NGZ));

    const int tid = threadIdx.x;
    const int tr = tid / KC, tl = tid % KC;
    const int j = j0 + tr, k = k0 + tl;
    const bool active = j < g.ny && k < g.nz;
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
    auto dtdz = [&](int K) { return (K >= 0 && K < g.nz) ? (TC)(g.dt / coef64[K]) : TC(0); };

    const TC cfx = (TC)g.dtdx, cfy = (TC)g.dtdy, rdx = (TC)g.rdx, rdy = (TC)g.rdy;
    const TC fz1 = (k > 0 && k < g.nz) ? (TC)(4.0 * coef64[6 * g.nz + k]) : TC(0);
    const TC fz2 = (k < g.nz - 1) ? (TC)(4.0 * coef64[7 * g.nz + k]) : TC(0);
    // B: the face below level k (K = k-1): exists for 1 <= k <= nz-1
    const bool zB = k >= 1 && k < g.nz;
    const TC cfBp = dtdz(k - 1), cfBn = dtdz(k);
    const bool farBp = k >= 2, farBn = k + 1 < g.nz;
    // C: warp 0: the y face north of row TJ-1; warp 1, lane r < TJ: the z face
    // above level k0+KC-1 of row r
    const int roleC = tid < KC ? 1 : (tid < KC + TJ ? 2 : 0);
    const int rC = tid - KC;  // row of a role-2 thread
    const int KT = k0 + KC - 1;
    const bool zC = KT < g.nz - 1;
    const TC cfCp = dtdz(KT), cfCn = dtdz(KT + 1);
    const bool farCn = KT + 2 < g.nz;

    const int oA = tr * KB + H + tl;             // A: phi rows j-2 .. j+1, v(j-1) one row down
    const int oB = (tr + 2) * KB + H + tl - 2;   // B: levels k-2 .. k+1 of row j; w(k-1)
    const int own = (tr + 2) * KB + H + tl;      // this thread's (j, k)
    const int oC = roleC == 1 ? TJ * KB + H + tl : (rC + 2) * KB + H + KC - 2;

    TO *out = reinterpret_cast<TO *>(set.out[sc]);
    TC ph[4] = {TC(0), TC(0), TC(0), TC(0)};  // phi at columns c-1 .. c+2 (own point)
    TC uw[3] = {TC(0), TC(0), TC(0)};         // u at columns c .. c+2
    TC D1 = TC(0), D2 = TC(0);                // y + z divergence of columns p-1, p-2
    TC Gx_w = TC(0);                          // x flux on the west face of the column written next

    for (int p = 0; p < nplanes; p++) {
        // every thread waits for plane p itself; the step's one CTA barrier
        // (after the face fluxes) shares the outcome
        const bool ok = pw_mbar_wait_bounded(&bars[p % NS], (uint32_t)((p / NS) & 1));
        TC *Gy = Gbuf + (p & 1) * (NGY + NGZ), *Gz = Gy + NGY;
        const TS *P = slot(p);
        const TS *Pu = P, *Pv = P + FS, *Pw = P + 2 * FS, *Pp = P + 3 * FS;
        const bool faces = p >= 2 && p < nplanes - 2;  // columns i0 .. i_end-1
        const TC pC = pw_to<TC>(Pp[own]);
        TC GA = TC(0), GB = TC(0);
        if (faces) {
            GA = pw_tvd_flux<TC>(pw_to<TC>(Pv[oA + KB]), cfy, cfy, pw_to<TC>(Pp[oA]), pw_to<TC>(Pp[oA + KB]), pC,
                                 pw_to<TC>(Pp[oA + 3 * KB]), true, true);
            if (zB)
                GB = pw_tvd_flux<TC>(pw_to<TC>(Pw[oB + 1]), cfBp, cfBn, pw_to<TC>(Pp[oB]), pw_to<TC>(Pp[oB + 1]),
                                     pC, pw_to<TC>(Pp[oB + 3]), farBp, farBn);
            if (roleC == 1) {
                Gy[TJ * KC + tl] = pw_tvd_flux<TC>(pw_to<TC>(Pv[oC + KB]), cfy, cfy, pw_to<TC>(Pp[oC]),
                                                   pw_to<TC>(Pp[oC + KB]), pw_to<TC>(Pp[oC + 2 * KB]),
                                                   pw_to<TC>(Pp[oC + 3 * KB]), true, true);
            } else if (roleC == 2) {
                Gz[rC * (KC + 1) + KC] =
                    zC ? pw_tvd_flux<TC>(pw_to<TC>(Pw[oC + 1]), cfCp, cfCn, pw_to<TC>(Pp[oC]), pw_to<TC>(Pp[oC + 1]),
                                         pw_to<TC>(Pp[oC + 2]), pw_to<TC>(Pp[oC + 3]), true, farCn)
                       : TC(0);
            }
            Gy[tr * KC + tl] = GA;
            Gz[tr * (KC + 1) + tl] = GB;
        }
        // own values of the newest plane
        ph[0] = ph[1];
        ph[1] = ph[2];
        ph[2] = ph[3];
        ph[3] = pC;
        uw[0] = uw[1];
        uw[1] = uw[2];
        uw[2] = pw_to<TC>(Pu[own]);
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
        TC D = TC(0);
        if (faces) D = (GA - Gy[(tr + 1) * KC + tl]) * rdy + fz1 * GB - fz2 * Gz[tr * (KC + 1) + tl + 1];
        if (p >= 3) {
            // x face between columns c = i0+p-4 and c+1: phi(c-1 .. c+2), u(c)
            const TC Gx = pw_tvd_flux<TC>(uw[0], cfx, cfx, ph[0], ph[1], ph[2], ph[3], true, true);
            if (p >= 4 && active) {
                const int i = i0 + p - 4;
                const TC s = (Gx_w - Gx) * rdx + D2;
                TO *o = out + (long long)(i + 2) * g.si + (long long)(j + 2) * g.sj + k;
                if (beta) {
                    if constexpr (std::is_same<TO, __nv_bfloat16>::value)
                        *o = __float2bfloat16_rn(__bfloat162float(*o) + (float)s);
                    else
                        *o = *o + (TO)s;
                } else {
                    if constexpr (std::is_same<TO, __nv_bfloat16>::value) *o = __float2bfloat16_rn((float)s);
                    else *o = (TO)s;
                }
            }
            Gx_w = Gx;
        }
        D2 = D1;
        D1 = D;
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
    const size_t smem = (size_t)NS * 4 * SH::FS * sizeof(TS) +
                        (size_t)2 * ((TJ + 1) * KC + TJ * (KC + 1)) * sizeof(TC) + NS * sizeof(uint64_t);
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
    g.ti = pw_pick_tile_i(m, tile_i, tiles, pw_slots(m, kern, TJ * KC, smem), 4);
    // the scalar and the k chunk are the fastest grid indices: the CTAs of one
    // tile run together and share the wind and the k-halo levels through L2
    dim3 grid((unsigned)(g.nkc * n), (unsigned)((m->ny + TJ - 1) / TJ), (unsigned)((m->nx + g.ti - 1) / g.ti));
    if (grid.y > 65535 || grid.z > 65535) return pw_fail(PW_ERR_SHAPE, "tvd: grid too large");
    kern<<<grid, TJ * KC, smem, st>>>(maps[0], maps[1], maps[2], set, m->coef64, g, beta, m->status);
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
