/*
 * pwadv.h -- C-ABI of a single-GPU (sm_103a) library that computes the
 * Piacsek-Williams (PW) advection source terms su, sv, sw of the wind fields
 * u, v, w of a large-eddy model: the computation the paper (a directive-based
 * hybrid of the Met Office NERC Cloud model) offloads to the GPU while the rest
 * of the dynamics runs on the CPU (sections 2.1 and 3; the scheme is the energy
 * conserving PW form named in section 3.1).
 *
 * Grid.  Arakawa C-grid, periodic in x and y, nx * ny columns of nz levels:
 *   u(i,j,k) at (x_{i+1/2}, y_j, zn_k), v(i,j,k) at (x_i, y_{j+1/2}, zn_k),
 *   w(i,j,k) at (x_i, y_j, zf_k), zf_k the top face of cell k.
 * w at the ground face (below k = 0) is 0, and the lid face w(.,.,nz-1) is 0 by
 * definition: the value stored there is never read and sw(.,.,nz-1) = 0 (for
 * nz = 1, where w is all lid, its values must be finite: they meet only zero
 * factors).
 *
 * Field layout.  Every field and source buffer holds (nx+4) * (ny+4) * nzp
 * elements: index ((i+2) * (ny+4) + (j+2)) * nzp + k for i in [-2, nx+2),
 * j in [-2, ny+2), k in [0, nzp); k is contiguous, x/y halos are 2 wide,
 * nzp >= nz is the padded column length given by pw_mesh_layout().  The library
 * never reads padding k >= nz.  Base pointers must be 16-byte aligned.
 *
 * Memory and streams.  Every pointer argument named a field or a source is a
 * DEVICE pointer owned by the caller.  The library owns meshes (coefficients,
 * status word, reduction scratch) and batches.  Unless stated otherwise a call
 * only enqueues work on `stream` (a cudaStream_t, NULL for the legacy default
 * stream) and returns without synchronising; errors found by argument checks are
 * returned at once, errors of the launch itself as PW_ERR_CUDA.
 *
 * Errors.  Every call returns a pw_status; pw_last_error() gives a thread-local
 * text for the last failing call of the calling thread.
 */
#ifndef PWADV_H
#define PWADV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PWADV_VERSION 1
/* Largest nz a mesh may have (columns are processed in k chunks above ~240). */
#define PW_MAX_NZ 4096

typedef enum {
    PW_OK = 0,
    PW_ERR_ARG = -1,      /* null pointer or value out of range */
    PW_ERR_SHAPE = -2,    /* sizes inconsistent with the mesh or beyond limits */
    PW_ERR_ALIGN = -3,    /* a buffer is not 16-byte aligned */
    PW_ERR_DTYPE = -4,    /* operation not available for the mesh dtype */
    PW_ERR_LID = -5,      /* pw_check_lid found a non-zero lid value */
    PW_ERR_CUDA = -6,     /* a CUDA runtime call failed (text in pw_last_error) */
    PW_ERR_TIMEOUT = -7,  /* a kernel gave up waiting for an asynchronous copy */
    PW_ERR_NOMEM = -8,    /* host or device allocation failed */
    PW_ERR_IO = -9,       /* the autotune cache file could not be read or written */
    PW_ERR_RANGE = -10    /* a value outside the range of PW_ALGO_F64_SPLIT (see there) */
} pw_status;

/* Storage type of the fields and sources of a mesh. */
typedef enum {
    PW_F64 = 0,   /* u, v, w and su, sv, sw in binary64; result within 1e-12 of FP64 */
    PW_F32 = 1,   /* binary32 storage and FP32 arithmetic */
    PW_BF16 = 2,  /* u, v, w in bfloat16; FP32 arithmetic; su, sv, sw in binary32 */
    PW_BF16_OUT = 3 /* u, v, w and su, sv, sw in bfloat16; FP32 arithmetic, each source
                       rounded once to bfloat16 (12 bytes per point instead of 18): error
                       within that of PW_BF16 plus 2^-8 |S| (the bfloat16 rounding).
                       Available for pw_advect, pw_advect_step, the scalar entry points,
                       pw_residuals, the halo fill and the host pipeline; the adjoint,
                       Euler and batched entry points return PW_ERR_DTYPE. */
} pw_dtype;

/* Arithmetic used for PW_F64 meshes (ignored for the other dtypes). */
typedef enum {
    PW_ALGO_AUTO = 0,       /* PW_ALGO_F64_SPLIT */
    PW_ALGO_F64_NATIVE = 1, /* FP64 instructions (the DP units of B300 are slow) */
    PW_ALGO_F64_SPLIT = 2   /* each double split exactly into two floats (scaled by 2^8),
                               products by FMA-exact FP32 transforms.  Error at each
                               point m:  |err| <= 1e-12 cond(m) + 2^-100 B(m) + 2^-140,
                               cond(m) = sum |c| |phi| (|a1| + |a2|) and B(m) =
                               sum |c| (|phi| + |a1| + |a2|) over the point's
                               elementary products c phi (a1 + a2); when every nonzero
                               input is at least 2^-40 in magnitude the first term
                               is the bound.  Range: |u|, |v|, |w| below 2^40 (about
                               1.1e12) and |theta|, |q| of the scalar entry points
                               below 2^60; a larger value, NaN or Inf is read as 0 and
                               sets PW_ERR_RANGE in the mesh status word
                               (pw_mesh_device_status): results that depend on it
                               carry no guarantee.  Nonzero values below 2^-110 are
                               read as 0 (within the bound).  The mesh coefficients
                               must have tcx, tcy, tzc1, tzc2, tzd1, tzd2 in
                               [2^-16, 2^8] and 0.25 rho_n, 0.25 rho_w in
                               [2^-36, 2^24] (checked by pw_mesh_create:
                               PW_ALGO_AUTO then uses native FP64, PW_ALGO_F64_SPLIT
                               returns PW_ERR_RANGE).  PW_ALGO_F64_NATIVE has none of
                               these limits. */
} pw_algo;

typedef struct {
    int nx, ny, nz;          /* interior points: nx, ny >= 1; 1 <= nz <= PW_MAX_NZ */
    double dx, dy;           /* horizontal spacing in m, > 0 */
    const double *dz;        /* HOST array of nz layer thicknesses (m), or NULL for
                                the geometric stretch dz(k) = 10 * 4^(k/(nz-1)) */
    const double *rho_n;     /* HOST, nz reference densities at cell centres, or NULL */
    const double *rho_w;     /* HOST, nz densities at the top faces, or NULL */
    double rho0, H_rho;      /* rho = rho0 exp(-z/H_rho) where not given; both 0 means
                                1.2 kg/m^3 and 8000 m; rho0 is also the ground density */
    pw_dtype dtype;
    pw_algo algo;
} pw_mesh_desc;

typedef struct pw_mesh pw_mesh;
typedef struct pw_batch pw_batch;

/* ---------------------------------------------------------------------------
 * Mesh: grid, coefficients and layout (the constants the paper copies to the
 * device once, at initialisation; section 3).
 * -------------------------------------------------------------------------*/

/* Create a mesh on the current CUDA device.  Computes, in FP64 on the GPU,
 *   zf(k) = sum_{m<=k} dz(m), zn(k) = zf(k) - dz(k)/2, dzn(k) = zn(k+1) - zn(k),
 *   rho_n, rho_w (given or rho0 exp(-z/H)), rho_w(-1) = rho0,
 *   tzc1(k) = 0.25 rho_w(k-1) / (rho_n(k) dz(k)),
 *   tzc2(k) = 0.25 rho_w(k)   / (rho_n(k) dz(k)),
 *   tzd1(k) = 0.25 rho_n(k)   / (rho_w(k) dzn(k)),   k < nz-1 (else 0),
 *   tzd2(k) = 0.25 rho_n(k+1) / (rho_w(k) dzn(k)),   k < nz-1 (else 0),
 *   tcx = 0.25/dx, tcy = 0.25/dy,
 * and FP32 copies of the vertical coefficients for the FP32/BF16 kernels.
 * Synchronises `stream`.  On success *out owns device memory; free it with
 * pw_mesh_destroy.  Returns PW_ERR_ARG / PW_ERR_SHAPE for bad descriptors. */
pw_status pw_mesh_create(const pw_mesh_desc *desc, void *stream, pw_mesh **out);

/* Free a mesh (NULL is allowed).  The caller must ensure no launch using it is
 * still running. */
void pw_mesh_destroy(pw_mesh *mesh);

/* Layout of every field/source buffer of this mesh, in ELEMENTS: nzp (padded
 * column length, a multiple of 8), stride_j = nzp, stride_i = (ny+4)*nzp, and
 * the total count (nx+4)*(ny+4)*nzp.  Any output pointer may be NULL. */
pw_status pw_mesh_layout(const pw_mesh *mesh, int64_t *nzp, int64_t *stride_j,
                         int64_t *stride_i, int64_t *total);

/* The arithmetic a PW_F64 mesh uses, with PW_ALGO_AUTO resolved: PW_ALGO_F64_SPLIT,
 * or PW_ALGO_F64_NATIVE when asked for or when the coefficients are outside the
 * split range (see pw_algo).  For the other dtypes PW_ALGO_AUTO is returned. */
pw_status pw_mesh_algo(const pw_mesh *mesh, pw_algo *out);

/* Copy the FP64 vertical grid to host memory `out` (12*nz doubles, in order
 * dz, zf, zn, dzn, rho_n, rho_w, tzc1, tzc2, tzd1, tzd2, W_uv, W_w where
 * W_uv = rho_n dz and W_w = rho_w dzn (0 on the lid face) are the energy
 * weights) and tcx, tcy into out_h[2] (may be NULL).  Synchronous. */
pw_status pw_mesh_coefficients(const pw_mesh *mesh, double *out, double *out_h);

/* Read (and with clear != 0 reset) the mesh's device status: 0; PW_ERR_TIMEOUT
 * when a kernel gave up waiting on an asynchronous copy since the last clear;
 * else PW_ERR_RANGE when a PW_ALGO_F64_SPLIT kernel met an input outside its
 * range (see pw_algo).  Both are sticky until cleared; a timeout also makes the
 * stencil kernels of this mesh return without work until it is cleared (an
 * out-of-range input does not).  Synchronises `stream`. */
pw_status pw_mesh_device_status(const pw_mesh *mesh, int clear, void *stream, int *status);

/* Failure-path self-test: launches a kernel that waits, with the library's
 * bounded mbarrier wait, for at most `cycles` clock cycles (1 .. 2e9) on a
 * barrier that nothing completes, and then records PW_ERR_TIMEOUT in the mesh
 * status word exactly as a stencil kernel that gave up on a copy would.  While
 * the word is set, stencil launches on the mesh return at once without work;
 * pw_mesh_device_status(clear = 1) resets it.  Faults nothing; for tests. */
pw_status pw_selftest_timeout(const pw_mesh *mesh, long long cycles, void *stream);

/* Tile configuration used by the stencil launches of this mesh: rows of
 * columns per CTA (tile_j, 1..32; fewer when a CTA would exceed 512 threads for
 * long columns) and columns marched per CTA along x (tile_i, >= 1; an upper
 * bound: launches shorten the march, down to 4 columns, while a small domain
 * would not fill the GPU).  Set by pw_autotune or by hand; not safe while
 * launches are being enqueued from another thread. */
pw_status pw_mesh_set_tile(pw_mesh *mesh, int tile_j, int tile_i);
pw_status pw_mesh_get_tile(const pw_mesh *mesh, int *tile_j, int *tile_i);

/* ---------------------------------------------------------------------------
 * Stencil entry points.
 * -------------------------------------------------------------------------*/

/* Periodic halo fill (the paper's halo swap at the start of a timestep,
 * section 2.1, on one device): copies interior columns into the 2-wide x and y
 * halos (corners included) of up to three fields of the mesh dtype, in place.
 * f1 must be non-NULL; f2, f3 may be NULL. */
pw_status pw_halo_periodic(const pw_mesh *mesh, void *f1, void *f2, void *f3, void *stream);

/* Adjoint of pw_halo_periodic: each halo value of up to three fields is ADDED
 * onto the interior value it is a periodic copy of, and the halo is set to 0.
 * Used to fold gradients that reached halo entries back onto the interior
 * degrees of freedom.  FP32 and FP64 meshes.  f2, f3 may be NULL. */
pw_status pw_halo_fold(const pw_mesh *mesh, void *f1, void *f2, void *f3, void *stream);

/* PW advection source terms (section 3.1): with halos of u, v, w filled,
 *  su = tcx [u(i-1)(u(i-1)+u(i)) - u(i+1)(u(i)+u(i+1))]
 *     + tcy [u(j-1)(v(i,j-1)+v(i+1,j-1)) - u(j+1)(v(i,j)+v(i+1,j))]
 *     + tzc1(k) u(k-1)(w(i,k-1)+w(i+1,k-1)) - tzc2(k) u(k+1)(w(i,k)+w(i+1,k))
 *  sv = tcx [v(i-1)(u(i-1,j)+u(i-1,j+1)) - v(i+1)(u(i,j)+u(i,j+1))]
 *     + tcy [v(j-1)(v(j-1)+v(j)) - v(j+1)(v(j)+v(j+1))]
 *     + tzc1(k) v(k-1)(w(j,k-1)+w(j+1,k-1)) - tzc2(k) v(k+1)(w(j,k)+w(j+1,k))
 *  sw = tcx [w(i-1)(u(i-1,k)+u(i-1,k+1)) - w(i+1)(u(i,k)+u(i,k+1))]
 *     + tcy [w(j-1)(v(j-1,k)+v(j-1,k+1)) - w(j+1)(v(j,k)+v(j,k+1))]
 *     + tzd1(k) w(k-1)(w(k-1)+w(k)) - tzd2(k) w(k+1)(w(k)+w(k+1)),  sw(nz-1) = 0,
 * terms whose face lies on the ground or the lid being 0.  Unlisted indices are
 * (i,j,k).  beta = 0 overwrites su, sv, sw; beta = 1 adds to them (dynamics
 * components add into shared source terms, section 3).  Only interior points
 * k < nz are written.  u, v, w are mesh dtype; su, sv, sw are binary64 for
 * PW_F64, bfloat16 for PW_BF16_OUT and binary32 otherwise.  Inputs and outputs
 * must not overlap. */
pw_status pw_advect(const pw_mesh *mesh, const void *u, const void *v, const void *w,
                    void *su, void *sv, void *sw, int beta, void *stream);

/* The forward Euler step fused into the stencil (the "step fields" integration
 * of section 3 done on the device, advection-only): with halos of u, v, w
 * filled,
 *   un = u + dt su(u,v,w),  vn = v + dt sv(u,v,w),  wn = w + dt sw(u,v,w)
 * on interior points k < nz, AND on their periodic halo images, so un, vn, wn
 * are ready for the next step without a halo fill; wn(nz-1) = 0 (the lid).
 * One pass: the fields are read once and the new state written once (the
 * separate pw_advect + pw_euler sequence moves 2.5 times the bytes).  un, vn,
 * wn have the mesh dtype (BF16 results are rounded to bf16).  The sources are
 * those of pw_advect (same accuracy); the update x + dt s is one FMA in the
 * compute precision.  No argument may alias another. */
pw_status pw_advect_step(const pw_mesh *mesh, const void *u, const void *v, const void *w,
                         void *un, void *vn, void *wn, double dt, void *stream);

/* Most scalars one pw_advect_scalars call advects. */
#define PW_MAX_SCALARS 16

/* PW advection of n cell-centred scalars (theta and the moisture / tracer
 * fields q: the further fields the advection component serves with the same
 * wind, section 3).  A scalar sits at the cell centre, so the wind on each face
 * of its cell is used as it is:
 *  s = hx [u(i-1) phi(i-1) - u(i) phi(i+1)] + hy [v(j-1) phi(j-1) - v(j) phi(j+1)]
 *    + hz1(k) w(k-1) phi(k-1) - hz2(k) w(k) phi(k+1)
 * with hx = 0.5/dx, hy = 0.5/dy, hz1(k) = 0.5 rho_w(k-1)/(rho_n(k) dz(k)),
 * hz2(k) = 0.5 rho_w(k)/(rho_n(k) dz(k)) (twice the momentum coefficients
 * tcx, tcy, tzc1, tzc2), w(-1) = 0 at the ground and w(nz-1) = 0 at the lid
 * (never read).  phi and sphi are HOST arrays of n device pointers (1 <= n <=
 * PW_MAX_SCALARS): phi[a] is a field of the mesh dtype and layout with its
 * halos filled (pw_halo_periodic), sphi[a] its source, binary64 for PW_F64,
 * bfloat16 for PW_BF16_OUT and binary32 otherwise; beta as in pw_advect.  Halos of u, v, w must be filled.
 * The wind is read once per group of scalars that fits a CTA's shared memory.
 * FP64 meshes compute in double-float arithmetic on the FP32 pipe (algo
 * PW_ALGO_F64_SPLIT, the default; same accuracy contract as pw_advect) or in
 * native FP64 (PW_ALGO_F64_NATIVE).  No output may alias an input or another
 * output. */
pw_status pw_advect_scalars(const pw_mesh *mesh, const void *u, const void *v, const void *w, int n,
                            const void *const *phi, void *const *sphi, int beta, void *stream);

/* The forward Euler step of the scalars fused into their stencil (the step-fields
 * update of section 3 on the device for theta and q): with halos filled,
 *   phin[a] = phi[a] + dt s(phi[a]; u, v, w)
 * on interior points and on their periodic halo images (ready for the next
 * step), s as in pw_advect_scalars, the update one FMA in the compute
 * precision.  phin[a] have the mesh dtype (BF16 results are rounded to bf16).
 * Same argument rules as pw_advect_scalars; dt must be finite. */
pw_status pw_advect_scalars_step(const pw_mesh *mesh, const void *u, const void *v, const void *w, int n,
                                 const void *const *phi, void *const *phin, double dt, void *stream);

/* The positivity-preserving scheme named beside PW (section 3.1, ULTIMATE;
 * section 4 sizes it at about sixteen times the PW work), for n cell-centred
 * scalars, in flux form on the C-grid:
 *  s = (u(i-1) f_x(i-1) - u(i) f_x(i)) / dx + (v(j-1) f_y(j-1) - v(j) f_y(j)) / dy
 *    + fz1(k) w(k-1) f_z(k-1) - fz2(k) w(k) f_z(k),
 *  fz1(k) = rho_w(k-1)/(rho_n(k) dz(k)), fz2(k) = rho_w(k)/(rho_n(k) dz(k)),
 * f_x(i) being the face value of phi on the face between cells i and i+1 where
 * u(i) sits (f_y, f_z alike); the ground face w(-1) and the lid w(nz-1) carry
 * no flux.  Face value (Leonard's ULTIMATE-QUICKEST): for velocity a, the
 * upwind cell C, the downwind cell D and the far-upwind cell U (one beyond C),
 * c = |a| dt / (width of C: dx, dy or dz(C)),
 *  q = (phi_C + phi_D)/2 - c (phi_D - phi_C)/2 - (1 - c^2)/6 (phi_D - 2 phi_C + phi_U),
 * held, where phi_C lies strictly between phi_U and phi_D, between phi_C and
 * min(phi_D, phi_U + (phi_C - phi_U)/c) in the direction of phi_D (the bound
 * toward phi_D applied first, so for c > 1 the face takes phi_C); elsewhere,
 * and where U would lie below the ground or above the lid, f = phi_C.
 * dt (> 0, finite) is the step the Courant numbers are taken for.  Halos of
 * u, v, w and of every phi[a] must be filled (the scheme reads two cells
 * along x and y).  phi and sphi are HOST arrays of n device pointers
 * (1 <= n <= PW_MAX_SCALARS) in the mesh layout; sphi[a] has the source type
 * of the mesh dtype (binary64 for PW_F64, bfloat16 for PW_BF16_OUT, binary32
 * otherwise); beta as in pw_advect.  Arithmetic: for PW_F64, double-float on
 * the FP32 pipe (PW_ALGO_F64_SPLIT, the default: the direction and
 * monotonicity decisions on exact FP64 differences, the rest within a few
 * units of 2^-46 of |a| (|phi_U| + |phi_C| + |phi_D|) per face; the range
 * contract of PW_ALGO_F64_SPLIT, out-of-range values setting PW_ERR_RANGE in
 * the mesh status) or native FP64 (PW_ALGO_F64_NATIVE); FP32 otherwise.  No output may alias an input or another
 * output.  Returns PW_ERR_ARG for bad arguments; timeouts as pw_advect. */
pw_status pw_advect_tvd(const pw_mesh *mesh, const void *u, const void *v, const void *w, int n,
                        const void *const *phi, void *const *sphi, double dt, int beta, void *stream);

/* ---------------------------------------------------------------------------
 * Fields in host memory: the step with its copies overlapped (the hybrid
 * offload of sections 3 and 3.1, where u, v, w go to the device every timestep
 * and the sources come back, asynchronously, to be integrated as they arrive).
 * -------------------------------------------------------------------------*/
typedef struct pw_pipeline pw_pipeline;

/* Called on a CUDA host thread once columns [i0, i1) of su, sv, sw are in the
 * host arrays; it must not call CUDA. */
typedef void (*pw_slab_fn)(void *user, int i0, int i1);

/* A pipeline for one mesh (which must outlive it): device copies of the six
 * fields (owned), three streams and per-slab events.  slab = x columns per
 * copy/compute unit (0: nx/32 rounded up).  Synchronises the device once. */
pw_status pw_pipeline_create(const pw_mesh *mesh, int slab, pw_pipeline **out);
void pw_pipeline_destroy(pw_pipeline *p);
/* slab width and number of slabs in use */
pw_status pw_pipeline_slab(const pw_pipeline *p, int *slab, int *nslab);
/* block the calling host thread until the last pw_advect_host has finished */
pw_status pw_pipeline_sync(pw_pipeline *p);
/* the six device copies u, v, w, su, sv, sw (library layout), e.g. to reuse
 * them with the device entry points; owned by the pipeline */
pw_status pw_pipeline_device_fields(const pw_pipeline *p, void **fields6);

/* The halo fill + PW step of pw_halo_periodic + pw_advect on HOST arrays in the
 * library layout: u, v, w (mesh dtype) in, su, sv, sw (source dtype) out
 * (beta = 1 adds to them, their old values travelling to the device too).
 * Only interior points (rows j < ny of columns i < nx, levels k < nz) of the
 * host arrays are read and written; host halos and padding levels are neither
 * read nor written.  Work proceeds in x-slabs: copy-in of slab s,
 * device halos, the stencil of slab s-1, copy-out of finished slabs, all on the
 * pipeline's own streams, ordered after the work already queued on `stream`;
 * `stream` then waits for the whole step, and the call returns without
 * blocking (except that, when on_slab was given to the previous call, it waits
 * for that call's callbacks to finish).  on_slab (may be NULL) is called, with
 * user, after each slab of the sources has reached the host.  Host arrays
 * should be page-locked (cudaHostAlloc / cudaHostRegister) for the copies to
 * overlap; pageable memory works but serialises them.  Inputs and outputs
 * must not overlap. */
pw_status pw_advect_host(pw_pipeline *p, const void *u, const void *v, const void *w, void *su, void *sv,
                         void *sw, int beta, pw_slab_fn on_slab, void *user, void *stream);

/* Device buffers in the pipeline for up to n scalars and their sources (1 <= n
 * <= PW_MAX_SCALARS; buffers already there are kept).  Synchronises the device. */
pw_status pw_pipeline_reserve_scalars(pw_pipeline *p, int n);

/* pw_advect_host with n cell-centred scalars advected by the same wind (theta
 * and q, which the paper's hybrid copies to the device only when the GPU is to
 * advect them): phi[a] (mesh dtype) and sphi[a] (source dtype) are HOST arrays
 * in the library layout; they travel, are halo-filled and advected slab by slab
 * with the wind (pw_advect_scalars), and on_slab follows each slab of all the
 * sources.  n = 0 is pw_advect_host.  Buffers for n scalars must have been
 * reserved (pw_pipeline_reserve_scalars). */
pw_status pw_advect_host_scalars(pw_pipeline *p, const void *u, const void *v, const void *w, void *su,
                                 void *sv, void *sw, int n, const void *const *phi, void *const *sphi,
                                 int beta, pw_slab_fn on_slab, void *user, void *stream);

/* Adjoint (transpose of the Jacobian of the map (u,v,w) -> (su,sv,sw) at the
 * given u, v, w) applied to incoming gradients gsu, gsv, gsw, with the periodic
 * halo fold included: gu, gv, gw receive gradients with respect to the INTERIOR
 * values (what the forward reads through a halo copy is added to the interior
 * point it copies):
 *   g = alpha * J(u,v,w)^T (gsu, gsv, gsw)            (beta = 0)
 *   g = g + alpha * J(u,v,w)^T (gsu, gsv, gsw)        (beta = 1)
 * Halos of u, v, w must be filled; the interior of gsu, gsv, gsw is read and
 * THEIR HALO COLUMNS ARE OVERWRITTEN with periodic copies.  gw(.,.,nz-1) = 0
 * (the lid is not a degree of freedom).  Only interior points k < nz of
 * gu, gv, gw are written.  For nz = 1 (sw identically 0) gsw is ignored and
 * overwritten with 0.  FP32 and FP64 meshes (FP64 in the mesh's arithmetic: double-float
 * on the FP32 pipe for PW_ALGO_F64_SPLIT, within its range, else native FP64);
 * PW_ERR_DTYPE for PW_BF16 and PW_BF16_OUT.  No argument may alias an output. */
pw_status pw_advect_adjoint(const pw_mesh *mesh, const void *u, const void *v, const void *w,
                            void *gsu, void *gsv, void *gsw,
                            void *gu, void *gv, void *gw, double alpha, int beta, void *stream);

/* Adjoint of one forward-Euler step x' = x + dt S(x) at the state x = (u,v,w):
 *   g_out = g_in + dt * J(u,v,w)^T g_in,
 * with the same halo conventions as pw_advect_adjoint (the halos of g_in are
 * overwritten; g_out(w lid) = 0).  Used for reverse sweeps over Euler loops. */
pw_status pw_euler_adjoint(const pw_mesh *mesh, const void *u, const void *v, const void *w,
                           void *gu_in, void *gv_in, void *gw_in,
                           void *gu_out, void *gv_out, void *gw_out, double dt, void *stream);

/* Forward-Euler step of the prognostic fields (the "step fields" integration of
 * section 3, advection-only): x <- x + dt * s for x in (u, v, w), s in
 * (su, sv, sw) on interior points k < nz, and the periodic halos of u, v, w are
 * refreshed in the same pass.  FP32 and FP64 meshes. */
pw_status pw_euler(const pw_mesh *mesh, void *u, void *v, void *w,
                   const void *su, const void *sv, const void *sw, double dt, void *stream);

/* Conservation diagnostics with FP64 accuracy, from a deterministic tree
 * reduction (a fixed grid of blocks whose records the last block to finish
 * adds in a fixed order: the order does not depend on timing, so repeated
 * calls give the same bits).  The reduction accumulates double-float sums on the FP32 pipe
 * (each sum within a few units of 2^-46 of the sum of its terms' magnitudes);
 * if an input is outside what that pass carries exactly (a nonzero |x| below
 * 2^-100 or from 2^56 up, NaN, Inf) or a sum of magnitudes is below 2^-40, the
 * sums are recomputed in plain FP64, so the result never depends on the range
 * of the data.  With weights
 * W = rho_n dz on u/v levels and rho_w dzn on w faces (lid face 0), for each
 * component c in (u, v, w) with source S:
 *   out[4c+0] = sum W phi S,   out[4c+1] = sum W |phi S|,
 *   out[4c+2] = sum W S,       out[4c+3] = sum W |S|,
 * so the energy residual is R_E = out[4c]/out[4c+1] (0 up to rounding for any
 * fields: the PW form conserves energy) and R_M = out[4c+2]/out[4c+3].
 * out is a HOST array of 12 doubles.  Synchronises `stream`.  Uses scratch that
 * the mesh owns, so concurrent calls on one mesh race. */
pw_status pw_residuals(const pw_mesh *mesh, const void *u, const void *v, const void *w,
                       const void *su, const void *sv, const void *sw, double *out,
                       void *stream);

/* The six conservation ratios from the twelve sums of pw_residuals (or
 * pw_residuals_noalloc): out[c] = R_E(c) = sums[4c] / sums[4c+1] and
 * out[3+c] = R_M(c) = sums[4c+2] / sums[4c+3] for c in (u, v, w), 0 where the
 * denominator is 0.  Host arrays; pure host arithmetic, no device work. */
pw_status pw_residual_ratios(const double *sums, double *out);

/* Largest nz accepted by pw_residuals_noalloc. */
#define PW_NOALLOC_MAX_NZ 4096

/* The conservation sums of pw_residuals for callers that cannot allocate
 * device memory when they need them -- e.g. because a caching allocator holds
 * all free device memory, or because an allocation inside a time-stepping loop
 * could synchronise the device -- and may not even hold a mesh (creating one
 * allocates).  The paper has no counterpart; this entry point exists for such
 * callers only.
 *
 * Arguments: the interior size nx, ny, nz and padded column length nzp of the
 * field layout (as pw_mesh_layout gives it; nzp a multiple of 8), the storage
 * dtype, the energy weights as HOST arrays of nz doubles (w_uv = rho_n dz on
 * u/v levels, w_w = rho_w dzn on w faces with the lid face 0; the last two
 * columns of pw_mesh_coefficients), the DEVICE buffers u, v, w, su, sv, sw
 * (16-byte aligned; sources binary64 for PW_F64, bfloat16 for PW_BF16_OUT,
 * binary32 otherwise) and a HOST
 * array out of 12 doubles, filled exactly as by pw_residuals.
 *
 * Allocation: none.  The only scratch is a file-scope device array of about
 * 127 KB, held on every GPU that loads the library until the process exits.
 * Every call looks up that array's device address (cudaGetSymbolAddress) with
 * the current device, so it stays right after a context is re-created; the
 * call synchronises `stream`, so it cannot sit inside a stream capture.  The six
 * buffers must be device (or managed) memory of the current device: anything
 * else returns PW_ERR_ARG before any launch.  nz above PW_NOALLOC_MAX_NZ returns
 * PW_ERR_SHAPE.  The
 * array is shared by every call: each call rewrites all of it that it reads, so
 * nothing depends on earlier contents, but calls that overlap on the GPU (on
 * different streams or host threads) race on it and must be serialised by the
 * caller.  Copies the weights in, runs the same FP64 reduction as
 * pw_residuals on `stream`, copies out and synchronises `stream`. */
pw_status pw_residuals_noalloc(int nx, int ny, int nz, int nzp, pw_dtype dtype,
                               const double *w_uv, const double *w_w,
                               const void *u, const void *v, const void *w,
                               const void *su, const void *sv, const void *sw,
                               double *out, void *stream);

/* Return PW_ERR_LID if any lid value w(i,j,nz-1) (interior) is not 0, else
 * PW_OK.  Synchronises `stream`. */
pw_status pw_check_lid(const pw_mesh *mesh, const void *w, void *stream);

/* ---------------------------------------------------------------------------
 * Batched ensembles: many independent subdomains (uneven sizes, own dx and dz)
 * advected in ONE persistent launch.
 * -------------------------------------------------------------------------*/

/* Create a batch over n PW_F32 meshes (each its own nx, ny, nz, dx, dy, dz);
 * the meshes must outlive the batch.  Device tables are built on `stream` and
 * the call synchronises it. */
pw_status pw_batch_create(pw_mesh *const *meshes, int n, void *stream, pw_batch **out);
void pw_batch_destroy(pw_batch *batch);

/* Bind member field buffers: host arrays of n device pointers each.  Copies the
 * member descriptors to the device and synchronises `stream`; after this,
 * pw_advect_batched enqueues a single kernel with no host-to-device copy and can
 * be captured in a CUDA graph.  Halos of every member must be filled before an
 * advect. */
pw_status pw_batch_set_fields(pw_batch *batch, void *const *u, void *const *v, void *const *w,
                              void *const *su, void *const *sv, void *const *sw, void *stream);

/* su, sv, sw of every member (same formulas as pw_advect) in one launch.  CTAs
 * pull tiles from a device work counter that this call resets on `stream`. */
pw_status pw_advect_batched(pw_batch *batch, int beta, void *stream);

/* Tile configuration of the batched launch: CTA size (threads, a multiple of 32
 * in 32..512; each member's tile has threads / (ceil(nz/4)) rows) and columns
 * marched per tile (tile_i).  Rebuilds the device tables; synchronises
 * `stream`.  On failure the previous configuration stays in force. */
pw_status pw_batch_set_tile(pw_batch *batch, int threads, int tile_i, void *stream);

/* Tile schedule of pw_advect_batched: persistent = 1 (default) launches
 * SMs x occupancy CTAs that pull tiles from a device counter; persistent = 0
 * launches one CTA per tile (the hardware scheduler hands them out in the same
 * longest-first order).  pw_batch_autotune tries both. */
pw_status pw_batch_set_schedule(pw_batch *batch, int persistent, void *stream);

/* Periodic halo fill of the bound u, v, w of every member in one launch. */
pw_status pw_batch_halo(pw_batch *batch, void *stream);

/* Read (and with clear != 0 reset) the batch's device status word (0 or
 * PW_ERR_TIMEOUT; sticky like the mesh status).  Synchronises `stream`. */
pw_status pw_batch_status(pw_batch *batch, int clear, void *stream, int *status);

/* ---------------------------------------------------------------------------
 * Tile autotuner (tile shapes chosen by timing candidates on the device).
 * -------------------------------------------------------------------------*/

/* Time each candidate tile (tile_j, tile_i) with pw_advect on the given buffers
 * (their contents are overwritten in su, sv, sw only), keep the fastest in the
 * mesh, and, if cache_path is not NULL, record it in a text cache keyed by
 * (nx, ny, nz, dtype, algo, SM count) -- a later call with the same key reads
 * the cache instead of timing.  Synchronises `stream`. */
pw_status pw_autotune(pw_mesh *mesh, const void *u, const void *v, const void *w,
                      void *su, void *sv, void *sw, const char *cache_path, void *stream,
                      float *best_ms);

/* Same for a batch whose fields are bound: picks one tile shape per size class
 * of members (by nz) and the persistent grid size. */
pw_status pw_batch_autotune(pw_batch *batch, const char *cache_path, void *stream, float *best_ms);

/* ---------------------------------------------------------------------------
 * Errors and version.
 * -------------------------------------------------------------------------*/
const char *pw_status_string(pw_status status);
const char *pw_last_error(void);
int pw_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PWADV_H */
