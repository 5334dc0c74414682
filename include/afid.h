/*
 * afid.h -- C ABI of the GB300 pressure-correction library (libafid.so).
 *
 * The library computes the data-parallel hot path of the fractional-step
 * solver of AFiD-GPU (Zhu et al., arXiv 1705.01423): the divergence of a
 * staggered velocity field, a real-to-complex FFT along x and a complex FFT
 * along y, one tridiagonal (Thomas) solve per wavenumber pair along the
 * stretched wall-normal direction z with zero-flux walls, the inverse FFTs, the
 * projection of the velocity and the pressure update (Sec. 2.2), and around it
 * the explicit terms and Crank-Nicolson wall-normal sweeps of one low-storage
 * RK3 substep (Sec. 2.1).
 *
 * Coordinates: x and y periodic and uniform, z bounded and stretched (the
 * paper calls the wall-normal direction x). All field arrays are C-ordered
 * [z][y][x] (x fastest), FP64, contiguous, resident on the CUDA device, and at
 * least 16-byte aligned:
 *   u, v, p, phi, rhs   [nz][ny][nx]    u on x-faces, v on y-faces, p/phi at centres
 *   w, T                [nz+1][ny][nx]  z-faces; planes 0 and nz are the walls
 *
 * Ownership: the caller owns every field buffer passed in; the context owns its
 * workspace, allocated once in afid_create and never inside a compute call.
 *
 * Execution: every compute call only enqueues work on the context's stream
 * and returns; it never synchronises the device, except that a non-NULL
 * afid_info* makes the call wait for its own work and fill the struct.
 * Arguments are validated on the host before anything is launched; a
 * validation error launches nothing. No call traps or spins on the device.
 *
 * Thread safety: one context must not be used from two host threads at once.
 */
#ifndef AFID_H
#define AFID_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AFID_OK = 0,
  AFID_ERR_INVALID_ARG = 1,      /* NULL pointer, bad index, non-positive length ...      */
  AFID_ERR_UNSUPPORTED_SIZE = 2, /* nx, ny not of the form 2^a 3^b 5^c, nx not a multiple
                                    of 16 or ny of 8, either > 4096; nz < 3 or > 4096   */
  AFID_ERR_ALIGNMENT = 3,        /* a device pointer not 16-byte aligned                  */
  AFID_ERR_NOT_CONVERGED = 4,    /* mixed refinement hit refine_max_iter (phi is the best) */
  AFID_ERR_INCONSISTENT_RHS = 5, /* |weighted mean of rhs| > 1e-8 max|rhs| (reported only
                                    when afid_info is requested; the mean is removed)     */
  AFID_ERR_CUDA = 6,             /* a CUDA runtime call failed                            */
  AFID_ERR_OOM = 7,              /* workspace allocation failed in afid_create            */
  AFID_ERR_TIMEOUT = 8           /* a bounded wait inside a kernel (TMA tile copy) gave
                                    up; reported by the next call that fills afid_info;
                                    the results of the calls since the last check are
                                    not valid                                             */
} afid_status;

typedef enum {
  AFID_FP64 = 0, /* every stage in FP64                                                  */
  AFID_MIXED = 1 /* FP32 transforms and Thomas sweeps, FP64 lowest modes, FP64 residual
                    iterative refinement of the Poisson solve                          */
} afid_precision;

/* flags */
#define AFID_POISSON_ONLY 1 /* do not allocate the RK3 substep workspace */
#define AFID_WARP_TRIDIAG 2 /* FP64: solve every (kx, ky) system with the warp-partitioned
                               solver (chunked Thomas per lane + parallel cyclic reduction
                               across the warp) instead of one system per thread -- the
                               variant for long wall-normal columns and few modes. Without
                               this flag or AFID_THREAD_TRIDIAG the context chooses: the
                               warp-partitioned solver when nz >= 256 and there are at most
                               64 systems (nx/2 + 1) ny per SM (measured on GB300: 3.2x
                               faster at 64 x 64 x 1296, 7.6x at 32 x 32 x 2048, even at
                               128 x 128 x 1296), one system per thread otherwise */
#define AFID_THREAD_TRIDIAG 16 /* FP64: always one system per thread */
#define AFID_NO_TMA 4       /* mixed: use the plain y-transform kernel (per-block loads into
                               padded shared memory) instead of the TMA-staged persistent
                               one for the FP32 passes (FP64 always uses the plain one) */
#define AFID_FUSE_SMALL_NZ 8 /* mixed, small nz: run the forward y transform, the solves of
                               every (kx, ky) and the inverse y transform in one kernel per kx
                               column (family yfft_thomas), the brick of the column, its pivots
                               and its low modes held in shared memory, wherever they fit and
                               the FP32 spectral array fits in half the L2. Without this flag
                               or AFID_NO_FUSE the context fuses where it was measured faster
                               on GB300: nz ny <= 8192 and ny <= 512 (the three stages 1.4-2.1x
                               faster, e.g. 0.13 against 0.28 ms at 512 x 512 x 8); at larger
                               bricks (512 x 512 x 32, 1024 x 1024 x 8) the fused kernel, one
                               block per SM, is 10% slower than the separate passes */
#define AFID_NO_FUSE 32     /* mixed: never fuse (the separate y-transform and Thomas passes) */

typedef struct {
  int nx, ny, nz;          /* cells; nx, ny = 2^a 3^b 5^c (the FFT radices 8/4/2/3/5),
                              nx a multiple of 16, ny of 8 (the paper's grids, e.g.
                              384, 768, 1280, are of this form)                     */
  double lx, ly;           /* periodic box lengths                                   */
  const double* zf;        /* HOST pointer, nz+1 face coordinates, strictly increasing */
  int precision;           /* afid_precision                                         */
  double refine_tol;       /* mixed: stop when the estimated relative error of phi
                              is <= refine_tol (see afid_info.err_estimate)          */
  int refine_max_iter;     /* mixed: maximum refinement iterations (>= 1)             */
  int flags;               /* OR of the AFID_* flags above, or 0                     */
} afid_grid_desc;

typedef struct {
  double nu, kappa;        /* momentum and scalar diffusivities                      */
  double buoyancy;         /* coefficient of T in the w equation                     */
  double u_bot, u_top;     /* wall velocities along x (Couette)                      */
  double T_bot, T_top;     /* wall temperatures                                      */
} afid_phys;

typedef struct {
  int iters;               /* refinement iterations used (1 for AFID_FP64)           */
  double rel_residual;     /* mixed: ||r||_2/||b - mean||_2 of the FP64 residual
                              computed before the last correction (||r||^2 summed
                              from its FP32 rounding; the norms are only
                              accumulated when afid_info is requested); FP64: 0     */
  double rhs_mean;         /* cell-volume-weighted mean removed from the rhs         */
  double rhs_absmax;       /* max |rhs|                                              */
  double max_div;          /* afid_project / substep: max |D u| after projection     */
  double err_estimate;     /* mixed: estimated relative error of phi (stopping rule:
                              ||d_k||^2/||d_{k-1}|| <= refine_tol ||phi|| for k >= 3,
                              ||d_2|| <= refine_tol ||phi|| at k = 2, d_k the k-th
                              correction, ||phi|| ~ ||d_1||); FP64: 0                */
} afid_info;

typedef struct afid_ctx afid_ctx;

/* Create a context for one grid on the current CUDA device. `stream` is a
 * cudaStream_t (NULL = legacy default stream). Allocates all workspace
 * (afid_workspace_bytes) and precomputes the metric, the twiddle tables and
 * the Thomas factor table of every wavenumber pair. Returns AFID_ERR_OOM if
 * the device cannot hold the workspace. Sec. 2.2 (workspace reuse: Sec. 3.3). */
afid_status afid_create(const afid_grid_desc* desc, const afid_phys* phys, void* stream,
                        afid_ctx** out);
afid_status afid_destroy(afid_ctx* ctx);
afid_status afid_set_stream(afid_ctx* ctx, void* stream);
size_t afid_workspace_bytes(const afid_grid_desc* desc);

/* Poisson solve, Sec. 2.2: phi with L phi = rhs - mean_W(rhs), mean_W(phi) = 0,
 * where L is the 7-point Laplacian of the staggered grid (periodic x, y; zero
 * flux at the walls) and mean_W the cell-volume-weighted mean. Forward
 * real-to-complex FFT in x, complex FFT in y, one Thomas solve per (kx, ky)
 * with modified wavenumbers 4 sin^2(pi k/N)/h^2, exact integration of the
 * singular (0,0) mode, inverse FFTs. rhs and phi: device [nz][ny][nx]; they
 * may alias. In AFID_MIXED the solve is FP32 with FP64 residual refinement. */
afid_status afid_poisson_solve(afid_ctx* ctx, const double* rhs, double* phi, afid_info* info);

/* Pressure correction, Sec. 2.1 and the last paragraph of Sec. 2.2: with
 * b = D(u)/s, phi = L^-1 b, then u -= s G_x phi, v -= s G_y phi,
 * w -= s G_z phi on interior z-faces, p += phi - beta dzz phi. The divergence
 * is fused into the forward x-transform. u, v, p: [nz][ny][nx]; w:
 * [nz+1][ny][nx], updated in place. s > 0. info->max_div is measured after the
 * projection when info is non-NULL. */
afid_status afid_project(afid_ctx* ctx, double* u, double* v, double* w, double* p, double s,
                         double beta, afid_info* info);

/* CFL number of Listing 1: max over cells of 0.5(|u_i+u_i+1|/dx +
 * |v_j+v_j+1|/dy + |w_k+w_k+1|/dzc_k), floored at 1e-8. Writes one double to
 * the DEVICE pointer cflm_dev, and dt = min(cfl/cflm, dt_max) to the context's
 * device-resident time step used by afid_rk3_substep when it is given dt <= 0. */
afid_status afid_cfl(afid_ctx* ctx, const double* u, const double* v, const double* w,
                     double cfl, double dt_max, double* cflm_dev);

/* One low-storage RK3 / Crank-Nicolson substep l in {0,1,2}, Sec. 2.1:
 * H = -A(u) + nu (dxx+dyy) q (+ buoyancy T on w), R = dt[gamma_l H + rho_l
 * Hprev - alpha_l G p + alpha_l nu dzz q], (I - beta_l dzz) dq = R with
 * beta_l = alpha_l dt nu/2 (kappa for T), q += dq, then the pressure
 * correction with s = alpha_l dt. gamma = (8/15, 5/12, 3/4), rho = (0, -17/60,
 * -5/12), alpha = gamma + rho. H* arrays are in/out: on entry the previous
 * substep's explicit terms (unused when l = 0), on exit this substep's. T and
 * HT may both be NULL (no scalar); T non-NULL with HT NULL makes T supply only
 * the buoyancy of the w equation, unchanged by the call (the temperature is
 * then advanced elsewhere, e.g. on the refined grid of afid_mr_*). dt <= 0
 * uses the device-resident dt set by afid_cfl. */
afid_status afid_rk3_substep(afid_ctx* ctx, int l, double dt, double* u, double* v, double* w,
                             double* T, double* p, double* Hu, double* Hv, double* Hw,
                             double* HT, afid_info* info);

/* max |D u| over all cells (divergence of Sec. 2.2 step 1) into a DEVICE double. */
afid_status afid_max_divergence(afid_ctx* ctx, const double* u, const double* v, const double* w,
                                double* out_dev);

/* Wall-normal statistics (the statistics of Sec. 3.2, accumulated only along
 * the wall-normal direction; the Nusselt number of Sec. 5 and the friction
 * velocity / friction Reynolds number of Sec. 5, Table 4).
 * profiles (HOST, may be NULL): [nz+1][AFID_STAT_NQ] horizontal means,
 *   0 <u>  1 <v>  2 <u^2>  3 <v^2>            on cell planes k = 0..nz-1 (row nz: 0)
 *   4 <w>  5 <w^2>  6 <T>  7 <T^2>  8 <w T>   on face planes k = 0..nz (6-8: 0 without T)
 * out (HOST, may be NULL): the scalars below, with H = zf[nz] - zf[0], Delta T =
 * T_bot - T_top and h = H/2 from the context's afid_phys:
 *   nu_volume  1 + <w T>_V / kappa (kappa = 1/sqrt(Ra Pr): Nu = 1 + sqrt(Ra Pr)<w T>_V),
 *              <.>_V over interior faces weighted by dzf;
 *   nu_bottom  -(<T>_1 - <T>_0) / dzc_0 / Delta T, nu_top likewise at the top wall
 *              (conductive flux through the wall cells);
 *   tau_bottom nu (<u>_0 - u_bot) / (dzc_0 / 2), tau_top nu (u_top - <u>_{nz-1}) /
 *              (dzc_{nz-1} / 2) (wall value half a cell away, as in the viscous term);
 *   re_tau     h u_tau / nu, u_tau = sqrt((|tau_bottom| + |tau_top|) / 2);
 *   ke         <(u^2 + v^2 + w^2) / 2>_V (u, v weighted by dzc, w by dzf).
 * u, v, w, T: device fields as in afid_rk3_substep (T may be NULL). The sums are
 * FP64 in a fixed order (deterministic). The call synchronises the context's
 * stream. */
#define AFID_STAT_NQ 9
typedef struct {
  double nu_volume, nu_bottom, nu_top;
  double tau_bottom, tau_top, re_tau;
  double ke;
} afid_stats;
afid_status afid_statistics(afid_ctx* ctx, const double* u, const double* v, const double* w,
                            const double* T, double* profiles, afid_stats* out);

/* Volume-averaged Nusselt number, the objective of the adjoint rollout (the
 * Nusselt number of Sec. 5, Table 3, in its volume form):
 *   Nu = 1 + coef <w T>_V,  <w T>_V = sum over interior z-faces k = 1..nz-1 of
 *        dx dy dzf_k w T / V,  V = lx ly (zf[nz] - zf[0]),
 * coef = sqrt(Ra Pr) in free-fall units (1/kappa). w, T: device [nz+1][ny][nx].
 * gw, gT (device [nz+1][ny][nx], either may be NULL): set to the derivatives
 * dNu/dw = coef dx dy dzf_k T / V and dNu/dT = coef dx dy dzf_k w / V on the
 * interior faces and zero on the walls -- the cotangent seeds of the adjoint.
 * nu_out (HOST, may be NULL): Nu; when given, the call synchronises the
 * context's stream. The sums are FP64 in a fixed order (deterministic). */
afid_status afid_nusselt(afid_ctx* ctx, const double* w, const double* T, double coef,
                         double* nu_out, double* gw, double* gT);

/* Transpose of the linear map rhs -> phi of afid_poisson_solve (exact
 * transpose: grhs = W_c solve(W_c^-1 gphi), W_c the cell volumes). gphi and
 * grhs: device [nz][ny][nx]; may alias. Always FP64. */
afid_status afid_poisson_solve_adjoint(afid_ctx* ctx, const double* gphi, double* grhs);

/* Transpose of the linear map (u, v, w, p) -> afid_project(u, v, w, p, s, beta).
 * On entry gu, gv, gw, gp hold the cotangents of the outputs; on exit the
 * cotangents of the inputs (in place). Always FP64. */
afid_status afid_project_adjoint(afid_ctx* ctx, double* gu, double* gv, double* gw, double* gp,
                                 double s, double beta);

/* Transpose of the Jacobian of afid_rk3_substep at the forward input
 * (u, v, w, T) (device, unchanged), with the same l and dt (dt must be > 0;
 * the adjoint treats dt as a constant). On entry g* hold the cotangents of the
 * substep's outputs (u, v, w, T, p, Hu, Hv, Hw, HT); on exit the cotangents of
 * its inputs (u, v, w, T, p, Hprev_u, ..., Hprev_T), in place. T/gT/gHT may be
 * NULL together. */
afid_status afid_rk3_substep_adjoint(afid_ctx* ctx, int l, double dt, const double* u,
                                     const double* v, const double* w, const double* T,
                                     double* gu, double* gv, double* gw, double* gT, double* gp,
                                     double* gHu, double* gHv, double* gHw, double* gHT);

/* ---- Multiple-resolution temperature grid (Sec. 6, conclusions and future
 * plans: the temperature on a grid finer than the momentum's, advanced with
 * its own refined time step; the paper leaves the details to a cited paper,
 * so the definitions below are this library's).
 *
 * Fine grid: every cell of the context's grid split into rx x ry x rz equal
 * cells; fine face zf_f[rz k + m] = zf[k] + (zf[k+1] - zf[k]) m / rz, so coarse
 * face k is fine face rz k. Fine fields are C-ordered like the coarse ones
 * with (nxf, nyf, nzf) = (rx nx, ry ny, rz nz): velocity uf, vf [nzf][nyf][nxf],
 * wf and the temperature Tf [nzf+1][nyf][nxf] (Tf planes 0 and nzf hold the
 * wall temperatures and are not changed).
 * Prolongation P: each velocity component is linear along each direction
 * between its coarse staggered samples, evaluated at its fine staggered
 * positions (periodic in x, y; along z, u and v reach their wall values u_bot /
 * u_top and 0 on the walls, w is linear between coarse faces).
 * Restriction R: coarse Tc[k][j][i] = mean of the rx x ry fine values of face
 * plane rz k over coarse cell (i, j).
 * Refined temperature step: the RK3/CN substep of afid_rk3_substep restricted
 * to the temperature equation, on the fine grid with the fine velocity.
 * All calls enqueue on the coarse context's stream; fine workspace (velocity,
 * explicit terms, right-hand side, two coarse velocity copies, Tc) is
 * allocated once by afid_mr_create. */
typedef struct afid_mr afid_mr;

/* 1 <= rx, ry, rz <= 8; the context must have the RK3 workspace (no
 * AFID_POISSON_ONLY). AFID_ERR_OOM if the fine workspace does not fit. The
 * refined grid refers to its context: destroy it before the context. */
afid_status afid_mr_create(afid_ctx* ctx, int rx, int ry, int rz, afid_mr** out);
afid_status afid_mr_destroy(afid_mr* mr);
afid_status afid_mr_dims(const afid_mr* mr, int* nxf, int* nyf, int* nzf);
size_t afid_mr_workspace_bytes(const afid_mr* mr);
/* The nzf+1 fine face coordinates into the HOST array zf_out. */
afid_status afid_mr_faces(const afid_mr* mr, double* zf_out);

/* Fine velocity at time t + theta dt: P((1 - theta) q0 + theta q1) for q = u,
 * v, w (coarse device fields; u1, v1, w1 may be NULL when theta = 0), 0 <=
 * theta <= 1, into the fine device fields uf, vf, wf. */
afid_status afid_mr_prolong(afid_mr* mr, const double* u0, const double* v0, const double* w0,
                            const double* u1, const double* v1, const double* w1, double theta,
                            double* uf, double* vf, double* wf);

/* Tc = R(Tf): Tf fine [nzf+1][nyf][nxf], Tc coarse [nz+1][ny][nx] (device). */
afid_status afid_mr_restrict(afid_mr* mr, const double* Tf, double* Tc);

/* Advances Tf from t to t + dt by n_sub >= 1 refined RK3/CN steps of dt / n_sub.
 * Substep l of refined step s uses the velocity at its start time, t + theta dt
 * with theta = (s + c_l) / n_sub, c = (0, 8/15, 2/3) (the partial sums of
 * alpha), linear in time between the coarse states (u0, v0, w0) at t and (u1,
 * v1, w1) at t + dt, prolonged. dt > 0 (host value). */
afid_status afid_mr_scalar_advance(afid_mr* mr, double dt, int n_sub, const double* u0,
                                   const double* v0, const double* w0, const double* u1,
                                   const double* v1, const double* w1, double* Tf);

/* One coupled step t -> t + dt: Tc = R(Tf); the three momentum substeps of
 * afid_rk3_substep (l = 0, 1, 2) with buoyancy from Tc, held for the step
 * (T non-NULL, HT NULL); then afid_mr_scalar_advance from the velocity at t to
 * the velocity at t + dt. u, v, w, p, Hu, Hv, Hw: coarse device fields as in
 * afid_rk3_substep (H* are scratch: substep 0 does not read them); Tf fine.
 * info, when non-NULL, is filled by the last momentum substep. */
afid_status afid_mr_step(afid_mr* mr, double dt, int n_sub, double* u, double* v, double* w,
                         double* p, double* Hu, double* Hv, double* Hw, double* Tf,
                         afid_info* info);

/* Wall-normal statistics of afid_statistics on the refined grid: the coarse
 * velocity (u, v, w, device) prolonged to the fine grid and the fine
 * temperature Tf (device) give the profiles (HOST, may be NULL,
 * [nzf+1][AFID_STAT_NQ]) and the scalars (HOST, may be NULL) with the fine
 * grid's metric, e.g. the Nusselt numbers of the refined temperature. The call
 * synchronises the context's stream. */
afid_status afid_mr_statistics(afid_mr* mr, const double* u, const double* v, const double* w,
                               const double* Tf, double* profiles, afid_stats* out);

/* Instrumentation: the FP64 operation rate this GPU delivers, measured. Every
 * FP64 stage of the path is bound by FP64 instruction issue on this part, so
 * this rate is the roofline denominator of those kernels. A kernel of
 * independent chains of dependent FP64 fused multiply-adds (eight per thread,
 * two 256-thread blocks per SM, `iters` FMAs per chain) runs on the context's
 * stream after a short warm-up launch and is timed with CUDA events; an FMA
 * counts as one operation. ops_per_s (HOST): FP64 operations per second;
 * ms_out (HOST, may be NULL): the timed launch in milliseconds. Synchronises
 * the stream. iters >= 1 (20000 runs about 20 ms on one GB300). */
afid_status afid_probe_fp64_rate(afid_ctx* ctx, int iters, double* ops_per_s, double* ms_out);

/* Test of the timeout path of the bounded device-side waits (the only waits
 * in this library: the TMA tile loads of the FP32 y transform). After this
 * call, the next TMA y-transform launch on the context runs block 0 with its
 * first tile stage armed for the tile's bytes but no copy issued, and a 1 ms
 * limit instead of 2 s: the block's wait runs out with nothing in flight for
 * that stage, it sets the fault flag, waits (bounded) for its other loads and
 * returns -- no fault and no hang. The next call that fills afid_info returns
 * AFID_ERR_TIMEOUT (the results of that solve are not valid) and clears the
 * flag; later calls on the context are unaffected. AFID_ERR_INVALID_ARG if the
 * context runs no TMA transform (FP64 contexts, AFID_NO_TMA, ny not a power of
 * two or > 2048). */
afid_status afid_test_tma_timeout(afid_ctx* ctx);

/* Last status text. */
const char* afid_status_string(afid_status s);

/* Number of kernels launched by this context since creation (instrumentation). */
long long afid_kernel_launches(const afid_ctx* ctx);

/* Instrumentation: when on, every launch group of the context is bracketed by
 * CUDA events on its stream, accumulated per kernel family (r2c_x, fft_y,
 * thomas, zero_mode, c2r_x, project, rhs, crank_nicolson, cfl_reduce, refine,
 * adjoint, cn_tables, mr_prolong, mr_scalar_rhs, mr_restrict, yfft_thomas; AFID_KERNEL_FAMILIES
 * of them; the afid_mr_* calls of a refined grid record into its coarse
 * context, their sweeps and tables under crank_nicolson and cn_tables). The first enable creates
 * the event pool (host-side CUDA events, no device memory). */
#define AFID_KERNEL_FAMILIES 16
afid_status afid_profile_enable(afid_ctx* ctx, int on);
/* Synchronises the stream and returns, per family, the milliseconds and the
 * number of launch groups recorded since the last read (arrays of n entries,
 * either may be NULL), then resets the counters. Returns AFID_ERR_INVALID_ARG
 * if the event pool overflowed (read more often). */
afid_status afid_profile_read(afid_ctx* ctx, double* ms, long long* launches, int n);
const char* afid_kernel_family_name(int family);

/* FP64 Poisson solve that allocates nothing. The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- code
 * that runs under a memory allocator it does not own (a host framework that
 * reserves the device memory pool), a real-time loop that must never
 * allocate, or a plugin that has no place to keep a context object. It
 * computes exactly what afid_poisson_solve computes in AFID_FP64 (same
 * kernels, same tables) for the grid (nx, ny, nz, lx, ly, zf_host), but
 * every piece of workspace -- metric, twiddles, wavenumbers, Thomas pivot
 * table and the spectral array -- lives in one file-scope __device__ array of
 * AFID_NOALLOC_BYTES (16 MiB) that every GPU loading the library holds until
 * the process exits. The rule is the byte count: the grid is accepted when
 *   16 nz ny roundup16(nx/2+1) + 8 nz (ny/2+1)(nx/2+1) bytes (the spectral
 *   array and the pivot table, each rounded up to 256 B) + the small tables
 *   (13 (nz+1) + 2 nx + 2 ny + nx/2 + ny/2 + 22 doubles, each rounded up to 256 B)
 * fit in AFID_NOALLOC_BYTES; e.g. 64^3, 128 x 128 x 64 and 128 x 128 x 80
 * fit, 256^3 does not. nx and ny must be powers of two here; a grid that does
 * not fit or is not of that form returns
 * AFID_ERR_UNSUPPORTED_SIZE before anything is launched. The caller passes
 * the input rhs and the output phi (device, [nz][ny][nx], 16-byte aligned; they
 * may alias) and a cudaStream_t. The call uploads the tables from a static
 * host staging buffer and launches on `stream`; it calls no cudaMalloc,
 * cudaFree or other allocating routine. Every call looks up the array's device
 * address (cudaGetSymbolAddress, which allocates nothing) for the device and
 * context current at that call, so a context change or a cudaDeviceReset
 * between calls leaves no stale address behind. The first call on a device
 * also loads the library's device code there: make that first call before
 * any stream capture. All calls share the one array and its contents persist
 * from the last call (every call rewrites the tables and the spectral array it
 * uses before reading them); calls that overlap on the GPU (two streams, two
 * host threads whose launches interleave) race on it. */
#define AFID_NOALLOC_BYTES (16u << 20)
afid_status afid_poisson_solve_noalloc(int nx, int ny, int nz, double lx, double ly,
                                       const double* zf_host, const double* rhs, double* phi,
                                       void* stream);

#ifdef __cplusplus
}
#endif
#endif /* AFID_H */
