/*
 * stagger.h - C ABI of libstagger, a GB300 (sm_103a) implementation of the
 * per-timestep right-hand side and low-storage RK3 step of the Stagger Code's
 * compressible MHD method (Stein, Nordlund, Collet & Trampedach, "The Stagger
 * Code for Accurate and Efficient, Radiation-Coupled MHD Simulations").
 *
 * Mesh and layout (Sect. "Centering"): a periodic nx*ny*nz box.  Every field
 * is one contiguous array of nx*ny*nz values indexed [k][j][i], x fastest.
 * rho and E (internal energy per volume, rho*e) sit at cell centres; the
 * momenta p = rho u and the magnetic field B on the lower cell faces
 * (px, Bx at (i-1/2, j, k), etc.).
 *
 * State: eight fields in the fixed order r, px, py, pz, E, Bx, By, Bz.  Each
 * is stored as an FP32 DEVIATION from a per-field FP64 constant ref[k]
 * (stagger_params.ref): the value used in the equations is ref[k] + stored.
 * Derivatives annihilate constants, so this is exact algebra; it keeps FP32
 * resolution for small perturbations on large backgrounds.
 *
 * Pointers: "device" arrays are caller-owned CUDA device memory of at least
 * nx*ny*nz floats (4-byte aligned); the library never frees them.  "host"
 * arrays are caller-owned host memory.  stream is a cudaStream_t passed as
 * void*; NULL means the legacy default stream.  Unless stated, calls are
 * asynchronous on that stream and return after enqueueing.
 *
 * Errors: every function returns STAGGER_OK (0) or a negative status and
 * never aborts or throws.  stagger_strerror() names a status.  A context is
 * not thread-safe: serialise calls that share one.
 */
#ifndef STAGGER_H
#define STAGGER_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  STAGGER_OK = 0,
  STAGGER_EINVAL = -1,      /* bad argument (NULL pointer, size, parameter)   */
  STAGGER_ECUDA = -2,       /* a CUDA runtime call failed                      */
  STAGGER_ENONFINITE = -3,  /* the state holds NaN/Inf (diagnostics, Courant)  */
  STAGGER_EOOM = -4,        /* device allocation failed                        */
  STAGGER_ETIMEOUT = -5,    /* reserved: a bounded device wait gave up         */
  STAGGER_EUNSUPPORTED = -6 /* not available on this entry (e.g. a stretched
                             * mesh in stagger_diagnostics_noalloc)         */
};

typedef struct stagger_ctx stagger_ctx;  /* opaque, library-owned */

typedef struct {
  int nx, ny, nz;          /* cells per axis, each >= 1; all axes periodic;
                            * ny, nz <= 65535 and nx*ny*nz < 2^31 (EINVAL)    */
  double dx, dy, dz;       /* uniform spacings, > 0 (dz is that of a uniform z;
                            * stagger_params.zc/zf give a stretched one)      */
} stagger_grid;

typedef struct {
  double gamma;            /* ideal-gas gamma, P = (gamma-1) E (&pde gamma)    */
  /* Richtmyer & Morton viscosity, eq. (RMnu): nu = nu1|u| + nu3 (c_s + c_A)
   * + nu2 dl_min max(0, -div u), spread by a 3-cell max and a 3-cell mean,
   * then nu_ii = dx_i <nu>, nu_ij = max(dx_i, dx_j) exp(interp ln<nu>),
   * eq. (nuij).  All zero and nu_const == 0 gives ideal MHD.                 */
  double nu1, nu2, nu3;
  double nu_const;         /* > 0: constant viscosity nu_ij = nu_const instead */
  double nuE;              /* energy diffusion factor, eq. (ediffuse)          */
  double nuB;              /* resistivity eta = nuB * nu (edge), eq. (ohm)     */
  double c1;               /* bulk term of eq. (itv); 0 typical                */
  int do_quench;           /* 1: quench stresses and eta J, eq. (quench)       */
  double qmax, qlim;       /* quench limits (&quench; 8 and 2)                 */
  int log_interp;          /* 1: rho to faces/edges as exp(interp ln rho)      */
  double Cdt, Cdtr, Cdtd;  /* Courant factors, eq. (courantcond) (0.4,0.1,0.7)*/
  double g[3];             /* constant gravity; source rho_face * g            */
  double ref[8];           /* per-field background added to the stored values */
  /* Newtonian cooling, eqs. (NewtonCool), (rhocool): dE/dt gains
   * -rho (e - e_cool) / t_cool * f(rho), e = E/rho, with f = 1 (cool_cut 0),
   * (rho/rho_cool)^2 / (1 + (rho/rho_cool)^2) (1, low-density cutoff) or
   * 1 / (1 + (rho/rho_cool)^2) (2, high-density cutoff).  t_cool = 0: off. */
  double t_cool, e_cool, rho_cool;
  int cool_cut;
  /* Smagorinsky viscosity, eq. (nusmag): dl_min * csmag * [2 (sum S_ii^2 -
   * (div u)^2 / 3 + sum_{i != j} S_ij^2)]^(1/2) is added to the Richtmyer &
   * Morton nu before its 3-cell max and mean, so nu_ii gains the
   * dx_i dl_min <...> form of eq. (nuij2).  0: off. */
  double csmag;
  /* Thread mapping of the fused FP32 kernels (no effect on the results beyond
   * rounding order).  0 (default): four consecutive x-cells per thread with
   * 16-byte loads and stores wherever nx % 4 == 0 and every array of the call
   * is 16-byte aligned, one cell per thread otherwise; 1: one cell per thread
   * everywhere.  Other values: STAGGER_EINVAL. */
  int scalar_cells;
  /* Second-order switch of the viscous stress (Sect. Equations, do_2nddiv):
   * where |D2_a ln rho| or |D2_a ln e| of a cell exceeds d2lnr_lim (D2_a f =
   * f(+1) - 2 f + f(-1) along axis a), every derivative along a in the strain
   * of eq. (itv), in its c1 div u term and in the viscous heating built from it
   * is the two-point difference instead of eq. (deriv).  0: off (default);
   * d2lnr_lim defaults to 0.3 (a negative limit flags every cell). */
  int do_2nddiv;
  double d2lnr_lim;
  /* Stretched vertical mesh (Sect. Derivatives; the mesh file of Sect. Input
   * and output): dz/dk at the cell centres (zc) and at the lower faces (zf),
   * nz positive values each, host arrays the caller owns, read (copied) by
   * stagger_create only.  z-derivatives are the index-space stencils times
   * 1/zc at centres and 1/zf at faces; the z diffusion length, dl_min of
   * eqs. (RMnu) and (nusmag) and the Courant limits use the local spacing;
   * diagnostics weight each cell by its spacing over the mean.  Both NULL
   * (default): uniform z of spacing grid.dz.  Needs nz > 1; one NULL and one
   * not, or a non-positive value: STAGGER_EINVAL. */
  const double* zc;
  const double* zf;
  /* Chromospheric cooling, eq. (ChromoCool): dE/dt gains
   * -rho (rho/rho_bot)^(5/3) (e - <e>) / t_chromo, <e> the mean of e = E/rho
   * over the horizontal plane (constant z) of the cell.  t_chromo = 0: off. */
  double t_chromo, rho_bot;
  /* Coronal optically thin cooling, eq. (CoronaCool): dE/dt loses
   * cor_L0 T^(-1/2) rho^2 exp(-(T / 10^4 K)^2) with T = cor_Tunit (gamma-1) e in
   * kelvin.  cor_L0 (the paper's constant over the squared atomic mass, in
   * code units) and cor_Tunit (kelvin per code unit) come from the caller's
   * unit system.  cor_L0 = 0: off. */
  double cor_L0, cor_Tunit;
  /* Kernel layout of the fluxes and divergences of one stage (no effect on
   * the results beyond rounding order).  0 (default): the fluxes are stored
   * to device arrays by one set of launches and differentiated, with the RK
   * update, by another; 1: one z-marching kernel forms every flux on chip
   * and applies the divergences and the update (uniform z only; a stretched z
   * keeps the default).  Other values: STAGGER_EINVAL. */
  int fuse_flux_div;
  /* The ratio of eq. (quench), q = |D2 T| / (M + |D2 T| / qmax), along each
   * axis the component is differentiated along.  quench_max3 0 (default): M =
   * |T| + quench_eps * max3|T|, the paper's point value, with the 3-cell max
   * of |T| along the axis weighted by quench_eps (default 1e-4) so that the
   * ratio is not 0/0 where T vanishes by symmetry on a grid point;
   * quench_max3 1: M = max3|T| alone.  quench_max3 outside {0, 1} or a
   * negative or non-finite quench_eps: STAGGER_EINVAL. */
  int quench_max3;
  double quench_eps;
  /* Closed walls along z (Sect. "Boundary Conditions", "Closed"), x and y
   * staying periodic.  zwalls 0 (default): z periodic.  zwalls 1: the
   * boundary points are the centre planes zghost and nz - 1 - zghost of the
   * arrays; the zghost planes beyond each are ghost planes, and the physical
   * fields are the centre planes zghost .. nz-1-zghost and the z faces
   * zghost+1 .. nz-1-zghost (p_z, B_z).  Every field is continued across a
   * boundary point by reflection about it with its parity: rho, E (so e),
   * p_x, p_y and B_z even, p_z, B_x and B_y odd (the paper's symmetric
   * parallel and anti-symmetric normal velocity, anti-symmetric parallel
   * field; B_z even keeps div B = 0); the odd centred fields are zero on the
   * boundary planes.  The library writes the ghost planes of the state it is
   * given (stagger_rhs, stagger_step, stagger_dt, stagger_courant,
   * stagger_diagnostics refill them before use, and a step leaves them
   * filled), zeroes those of a time derivative, takes the Courant step over
   * the physical planes only, and reports the totals the closed box
   * conserves (half weight on the boundary planes; sum p_z over the physical
   * faces).  zghost >= STAGGER_ZGHOST_MIN (the reach of the right-hand side)
   * and nz >= 2 zghost + 2, a uniform z, no Smagorinsky term (whose
   * strain-rate centring reaches three cells further) and zero ref[] of the
   * odd fields p_z, B_x, B_y (the reflection acts on the stored deviations),
   * else STAGGER_EINVAL.  The op-graph
   * entries (stagger_rhs_unfused*, stagger_step_unfused_f64,
   * stagger_step_adjoint*) and stagger_diagnostics_noalloc return
   * STAGGER_EUNSUPPORTED with closed walls.  Gravity along z acts on the physical
   * faces; a stratified atmosphere is not in balance at a wall under this
   * continuation (the density is reflected, not extrapolated).
   * zwalls 2: rigid walls (Sect. "Boundary Conditions", "Rigid") at the same
   * planes.  Every plane outside zghost .. nz-1-zghost is a ghost plane, for
   * the z-face fields too (so the faces zghost and nz-1-zghost are physical).
   * The ghost values of rho, E and B are the caller's and never change (their
   * time derivatives are zero); before every use of a state the library sets
   * its ghost momenta to p_d = rho_d u_d(b): the density at the p_d position
   * times the velocity p_d / rho_d of the boundary plane b at the same (x, y)
   * (b = zghost below, nz-1-zghost above).  The Courant step and the
   * diagnostics (plain sums) cover the physical planes.  The same zghost, nz,
   * uniform-z and no-Smagorinsky conditions hold; ref[] is unrestricted.
   * Ghost planes holding a hydrostatic atmosphere keep it in balance at the
   * wall.  With rigid walls stagger_rhs_unfused, stagger_rhs_unfused_f64 and
   * stagger_step_unfused_f64 apply the same fill and zero ghost derivatives;
   * the adjoint entries and stagger_diagnostics_noalloc return
   * STAGGER_EUNSUPPORTED. */
  int zwalls;
  int zghost;
  /* Energy diffusion of the fluctuations only, eq. (ediffav): with ediffav 1
   * (and a viscosity on) the diffusion flux of eq. (ediffuse) becomes
   * nuE dn(rho nu_ii) e dddn(ln e - ln <e>_h), <e>_h the mean of e = E/rho over
   * the horizontal plane (constant z) of the cell, e at the face by
   * interpolation.  0 (default): eq. (ediffuse).  Other values: EINVAL. */
  int ediffav;
  /* Pressure gradient of eq. (mom) through ln(P/P_aver), eq. (pressure) (Sect.
   * "Equations"): with lnp_aver 1 the pressure leaves the diagonal momentum
   * fluxes and the gradient along d at the d face is
   *   exp(dn_d ln P_aver + dn_d ln(P/P_aver)) (dddn_d ln(P/P_aver) + dddn_d ln P_aver),
   * P_aver the mean of P = (gamma - 1) E over the horizontal plane (constant z)
   * of the cell, of the state the right-hand side is evaluated on; the
   * derivative of ln P_aver vanishes for d = x, y.  0 (default): P in the
   * diagonal fluxes.  Other values, or lnp_aver 1 with fuse_flux_div 1:
   * STAGGER_EINVAL. */
  int lnp_aver;
  /* Stellar-atmosphere z boundaries (Sect. "Boundary Conditions", "Stellar
   * Atmosphere"), zwalls 3, at the planes of the closed walls: physical
   * centres zghost .. nz-1-zghost and z faces zghost+1 .. nz-1-zghost, every
   * other plane a ghost plane with zero time derivative.  The bottom (the
   * interior boundary) is the end gravity points to (g[2] < 0: the low
   * index end; g[2] == 0: STAGGER_EINVAL), the other end is the top.  Before
   * every use of a state its ghost planes are filled: ln rho and e = E/rho
   * extrapolated linearly from the boundary plane and its inner neighbour
   * (at the top the ghost density limited to [top_rho_lo, top_rho_hi] times
   * its plane mean, e to [e_b / top_e_fac, e_b top_e_fac] about the boundary
   * value); bottom momenta symmetric about the boundary point; top momenta
   * rho_d times the boundary velocity limited to |u| <= top_umax; B
   * extrapolated linearly and, at the bottom, its horizontal components
   * blended toward bdry_B (eq. bin) by f = 1/(1 + exp(U/bdry_u)) (eq.
   * smooth), U the outward velocity at the boundary (f -> 1 in inflows).
   * On the bottom plane dE/dt = (bdry_E - E)/bdry_t; d rho/dt = f (bdry_rho -
   * rho)/bdry_t + (1 - f)(F_rho + ((bdry_E - E)/bdry_t - F_E)/(gamma e)) (eqs.
   * rein, constS to addderiv for the ideal gas); the horizontal momenta
   * lose f (p_h - <p_h>)/bdry_t.  On the top plane the vertical mass-flux
   * divergence is replaced by the outward-signed flux over the pressure
   * scale height (gamma - 1) e / |g_z| (eq. rbdrylo).  bdry_E is internal
   * energy per volume.  The top field's relaxation toward the potential
   * field is top_tpot below.  Needs bdry_t, bdry_rho, bdry_E, bdry_u, top_umax > 0, 0 <
   * top_rho_lo <= 1 <= top_rho_hi, top_e_fac >= 1, nz >= 3 zghost + 2 (the
   * mirrored bottom momenta come from physical planes), fuse_flux_div 0 and
   * the conditions of the closed walls but the ref[] one, else
   * STAGGER_EINVAL.  stagger_rhs_unfused, stagger_rhs_unfused_f64 and
   * stagger_step_unfused_f64 apply the same fill and rates around the op
   * graph; the adjoint entries and stagger_diagnostics_noalloc return
   * STAGGER_EUNSUPPORTED. */
  double bdry_t, bdry_rho, bdry_E, bdry_u;
  double bdry_B[3];
  double top_rho_lo, top_rho_hi, top_e_fac, top_umax;
  /* With zwalls 3 and top_tpot > 0: the horizontal field of the top plane also
   * relaxes toward the potential field of its normal field (Sect. "Exterior
   * Boundary In the Atmosphere"): dB_h/dt += (B_pot,h - (B_h - <B_h>)) /
   * top_tpot, B_pot,h the horizontal components on the plane of the
   * current-free field that decays outward from B_z on the nearest inside z
   * face, by horizontal Fourier modes (B_h = -i s (k_h/|k|) B_z, s the outward
   * direction; no mean or Nyquist part).  0 (default): off.  Negative or not
   * finite, or nx > 24576 with it: STAGGER_EINVAL.  The op-graph entries return STAGGER_EUNSUPPORTED
   * with it. */
  double top_tpot;
} stagger_params;

/* Ghost planes needed at each closed z wall: the reach of the right-hand
 * side along an axis (14 cells with viscosity and the quench). */
#define STAGGER_ZGHOST_MIN 14

/* Fill *p with the defaults of the paper's namelists: gamma 5/3, ideal MHD,
 * nuE = nuB = 1, qmax 8, qlim 2 (quench_eps 1e-4), log_interp 1, Cdt 0.4, Cdtr 0.1, Cdtd 0.7,
 * no gravity, zero references, no cooling (rho_cool 1, rho_bot 1, cor_Tunit 1),
 * no second-order switch (d2lnr_lim 0.3), uniform z.  Returns STAGGER_EINVAL if p is NULL. */
int stagger_params_default(stagger_params* p);

/* Create a context for one grid and parameter set on the current CUDA device.
 * Allocates all device scratch once (about 30 fields of nx*ny*nz floats for
 * the fused step; more on the first adjoint call).  *out receives the handle.
 * Errors: EINVAL (bad grid/params/NULL), EOOM, ECUDA. */
int stagger_create(const stagger_grid* grid, const stagger_params* params,
                   stagger_ctx** out);

/* Release a context and all its device memory (synchronises the device).
 * NULL is accepted.  Returns OK or ECUDA. */
int stagger_destroy(stagger_ctx* ctx);

/* F(f): the eight time derivatives of eqs. (mass), (mom), (ien), (indu)
 * at the state, written to dfdt (8 device arrays, NOT deviations: the plain
 * derivative values).  state and dfdt must not overlap.  Async. */
int stagger_rhs(stagger_ctx* ctx, float* const state[8], float* dfdt[8], void* stream);

/* One full low-storage RK3 step, eqs. (ddt), (tupdate), (tconst), updating
 * the 8 device arrays of state in place.  dt > 0: that step; dt <= 0: the
 * Courant step of eq. (courantcond), taken from the state and its stage-1
 * derivative and held for all three stages (computed on the device; no host
 * synchronisation).  If dt_used is not NULL it is a HOST pointer: the call
 * then synchronises the stream and stores the step used.  Async otherwise. */
int stagger_step(stagger_ctx* ctx, float* state[8], double dt, double* dt_used, void* stream);

/* Run nsteps steps as stagger_step does, with dt <= 0 meaning Courant.
 * A Courant-mode step (dt <= 0) with per-kernel timing off is replayed from a
 * CUDA graph of its launches, captured on the first such call for the given
 * state arrays (on a private stream; launched on `stream`) and captured again
 * when the arrays change; stagger_step and stagger_step_host do the same. */
int stagger_run(stagger_ctx* ctx, float* state[8], int nsteps, double dt, void* stream);

/* The Courant step of eq. (courantcond) for this state (FP64 reduction on the
 * device).  Synchronises; *dt_host receives it, limits[3] (may be NULL) the
 * wave-speed, rate-of-change and diffusion limits (HUGE_VAL when inactive).
 * Returns ENONFINITE if the state produced a non-finite limit. */
int stagger_courant(stagger_ctx* ctx, float* const state[8], double* dt_host,
                    double limits[3], void* stream);

/* The same Courant step as an asynchronous call: out receives 4 doubles, dt
 * and the wave-speed, rate-of-change and diffusion limits (HUGE_VAL when
 * inactive).  on_device 1: out is a DEVICE pointer, written on the stream
 * with no host synchronisation (the value a later stagger_step with dt > 0
 * could be given after a device-to-host read, or a device-side consumer
 * reads directly); on_device 0: out is a HOST pointer and the call
 * synchronises, returning ENONFINITE for a non-finite step.  The step is
 * computed from the state and its stage-1 derivative, as stagger_step does
 * with dt <= 0.  Errors: EINVAL (NULL, on_device not 0 or 1), ECUDA. */
int stagger_dt(stagger_ctx* ctx, float* const state[8], double* out, int on_device, void* stream);

/* FP64 diagnostics of the state (plain sums over cells): out[0..9] =
 * sum r, sum px, sum py, sum pz, sum E, sum 1/2 p.u (faces), sum 1/2 B^2,
 * max |div B|, rms div B (div B = sum_i ddup_i B_i at centres), count of
 * non-finite values.  Values include the refs.  Synchronises.  Returns
 * ENONFINITE (after filling out) if the count is nonzero. */
int stagger_diagnostics(stagger_ctx* ctx, float* const state[8], double out[10], void* stream);

/* Adjoint of one fixed-dt step (vector-Jacobian product): given the step's
 * input state_n (deviations, as passed to stagger_step), its dt > 0 and the
 * cotangent lam_np1 of the output state, write the cotangent of the input
 * state to lam_n (8 device arrays, may alias lam_np1).  Recomputes the stage
 * states, then reverses the RK3 recurrence and the right-hand side.  The
 * first call allocates the reverse-sweep workspace (about 3 x the number of
 * graph nodes x nx*ny*nz floats).  Async. */
int stagger_step_adjoint(stagger_ctx* ctx, float* const state_n[8], double dt,
                         float* const lam_np1[8], float* lam_n[8], void* stream);

/* Unfused evaluation of the same right-hand side: the equations as a graph
 * of primitive staggered operations (eqs. (deriv), (interp) and pointwise
 * arithmetic), one launch per operation.  It is the forward of the adjoint's
 * reverse sweep and a cross-check of the fused path.  The first call
 * allocates one array of nx*ny*nz values per graph node (a few hundred).
 * _f64 variants take FP64 device arrays (deviations, as above) and compute
 * in FP64.  Async. */
int stagger_rhs_unfused(stagger_ctx* ctx, float* const state[8], float* dfdt[8], void* stream);
int stagger_rhs_unfused_f64(stagger_ctx* ctx, double* const state[8], double* dfdt[8],
                            void* stream);
/* One fixed-dt (dt > 0) RK3 step through the unfused graph in FP64, in place. */
int stagger_step_unfused_f64(stagger_ctx* ctx, double* state[8], double dt, void* stream);
/* stagger_step_adjoint in FP64 (FP64 device arrays). */
int stagger_step_adjoint_f64(stagger_ctx* ctx, double* const state_n[8], double dt,
                             double* const lam_np1[8], double* lam_n[8], void* stream);

/* End-to-end step through host memory: copies the 8 HOST arrays (pinned
 * recommended) to a library-owned device state, runs nsteps steps (dt <= 0:
 * Courant), and copies the result back into the same host arrays.
 * Synchronises.  The device copy is allocated on the first call. */
int stagger_step_host(stagger_ctx* ctx, float* state_host[8], int nsteps, double dt,
                      void* stream);

/* Per-kernel timing of the fused path with CUDA events recorded on the
 * launch stream around each launch.  on != 0 enables it (and clears the
 * totals), 0 disables it.  Returns OK or EINVAL. */
int stagger_timing(stagger_ctx* ctx, int on);

/* Collect the timing events (synchronises the stream) and report, for up to
 * max kernel kinds, the kernel name (static string), the summed device time
 * in milliseconds and the number of timed launches.  Any output array may be
 * NULL.  Returns the number of kernel kinds (>= 0) or a negative status. */
int stagger_kernel_times(stagger_ctx* ctx, int max, const char** names, double* total_ms,
                         long long* launches, void* stream);

/* Diagnostics without any allocation (the paper has no counterpart; this is
 * a library convenience).  Same outputs, status and synchronisation as
 * stagger_diagnostics, but it takes the grid and parameters directly instead
 * of a context and allocates nothing: no cudaMalloc, no cudaFree, no host heap.
 * Its scratch is a fixed 5 MiB array in the library's device image, which
 * every GPU that loads the library keeps until the process exits.  It is for
 * callers that cannot allocate: an application whose memory pool already
 * owns the device's memory, a monitoring tool that must not change the
 * footprint of the run it inspects, or code that has no context (creating
 * one allocates tens of arrays of the grid's size).
 * Limit: at most 65536 thread blocks of 32 x 2 x 4 cells, i.e.
 * ceil(nx/32) * ceil(ny/2) * ceil(nz/4) <= 65536 (for example 256^3); larger
 * grids return STAGGER_EINVAL.  A stretched z (params->zc, zf) needs its mesh
 * on the device and returns STAGGER_EUNSUPPORTED.  The grid and parameters
 * pass the same checks as stagger_create (STAGGER_EINVAL).  Every call that is
 * not being captured looks up the array's device address
 * (cudaGetSymbolAddress) on the current device, so a context torn down and
 * rebuilt (cudaDeviceReset) is safe; a call made during stream capture reuses
 * the address of the last uncaptured call on that device, and returns
 * STAGGER_EUNSUPPORTED if there was none: make the first call on each device
 * before any stream capture, and again after a device reset.  All calls share the one array:
 * calls that overlap on the GPU (two streams, two host threads) race, so
 * serialise them.  Each call overwrites every scratch entry it reads. */
int stagger_diagnostics_noalloc(const stagger_grid* grid, const stagger_params* params,
                                float* const state[8], double out[10], void* stream);

/* Number of cells nx*ny*nz of the context's grid (0 for NULL). */
size_t stagger_cells(const stagger_ctx* ctx);

/* Count of this library's kernels launched on ctx since creation. */
long long stagger_launch_count(const stagger_ctx* ctx);

/* Short English description of a status code (static storage). */
const char* stagger_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* STAGGER_H */
