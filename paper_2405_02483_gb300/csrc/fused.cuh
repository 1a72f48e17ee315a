// Fused FP32 stage kernels of the MHD right-hand side and the RK3 update.
#pragma once

#include <utility>
#include <vector>

#include "common.cuh"

namespace stg {

// Scalar parameters in the precision of the kernels.
struct KPar {
  float ih[3];          // 1/dx, 1/dy, 1/dz
  float r0, E0, e0;     // reference density, energy, e0 = E0/r0
  float Ec;             // E0 - e0 r0 (E0 when r0 = 0), so that e - e0 = (E' + Ec - e0 r') / (r' + r0)
  float pref[3], Bref[3];
  float gamma, gm1;
  int visc, rm;         // any viscosity; Richtmyer-Morton (else constant)
  float nu1, nu2dl, nu3, nu_const;
  float sp[3];          // diffusion length per axis
  float spp[3];         // max(sp) of edge pairs: [yz (Ex), zx (Ey), xy (Ez)]
  float nuE, nuB, c1, inv_qmax, qlim;
  int qmax3;            // quench ratio over the 3-cell max of |T| (else |T| + qeps max3|T|)
  float qeps;
  int log_interp, do_quench, r0pos;
  float g[3];
  float inv_tcool, e_cool, inv_rho_cool;   // Newtonian cooling (inv_tcool 0: off)
  int cool_cut;
  float csmag_dl;       // Smagorinsky constant times dl_min (0: off)
  int d2div;            // second-order switch of the stress derivatives
  float d2lim;          // its limit on |D2 ln rho|, |D2 ln e|
  float dlmin;          // dl_min of the mesh
  // Stretched z mesh (null when uniform): dz/dk at centres and lower faces
  // and their inverses (nz values each), the smallest active x, y spacing, and
  // the raw coefficients that multiply the local dl_min there.
  const float *hzc, *hzf, *jzc, *jzf;
  float dlxy, nu2, csmag;
  double izbar;         // 1 / mean dz/dk (diagnostic weights)
  float inv_tchromo, inv_rhobot;   // chromospheric cooling (0: off)
  const double* emean;  // plane means of e - e0, one per z (chromospheric cooling)
  float corL0, corTu;   // coronal thin cooling (corL0 0: off)
  // Closed z walls (reading R22): the physical centre planes are klo..khi,
  // the planes outside are ghost planes filled by reflection.
  int wall, klo, khi;
  int ediffav;          // energy diffusion of ln e - ln <e>_h, eq. (ediffav), R23
  // Pressure gradient through ln(P/P_aver), eq. (pressure), R24: the plane
  // means of E - E0 (nz), P_aver per centre plane, exp(dn_z ln P_aver) and
  // dddn_z ln P_aver per lower z face (nz floats each).
  int lnpa;
  const double* Emean;
  const float *pa, *paz, *dpaz;
  const float *qm, *qden;   // <E'> and E0 + <E'> per plane, for ln(P/P_aver) in k_lr_ed
  // Stellar-atmosphere z boundaries (R26, wall 3): the bottom and top boundary
  // planes and their outward index directions, 1/bdry_t, the bottom targets,
  // 1/bdry_u, B_bdry (x, y), the top limits, |g_z|, and the plane means: the
  // extrapolated density of the top ghost planes 1..zghost (zghost doubles),
  // the p_x and p_y deviations of the bottom plane, the B_x and B_y deviations
  // of the top plane.
  int obot, otop, osb, ost;
  float oinv_t, orho, oE, oinv_u, oBx, oBy, orlo, orhi, oefac, oumax, ogabs;
  const double* omean;
  // R27: 1/top_tpot (0: off) and the potential-field targets of the top
  // plane's B_x, B_y fluctuations (one plane each).
  float oinv_tpot;
  const float *bpx, *bpy;
};

// Fields of the fused path, one contiguous device array each.
enum Fld {
  F_LR = 0, F_UX, F_UY, F_UZ,                       // ln(rho/r0) (or rho'), face velocities
  F_NV, F_NM, F_NU, F_LNU,                          // raw, max, smoothed nu, ln<nu>
  F_TXX, F_TYY, F_TZZ, F_TXY, F_TYZ, F_TZX,         // stress tau
  F_RX, F_RY, F_RZ, F_JX, F_JY, F_JZ,               // eta J and J
  F_QXX, F_QYY, F_QZZ, F_QXY, F_QYZ, F_QZX,         // quenched tau
  F_EX, F_EY, F_EZ,                                 // total electric field (edges)
  F_WC, F_WX, F_WY, F_WZ,                           // heating densities (centre, edges)
  F_MXX, F_MYY, F_MZZ, F_MXY, F_MYX, F_MXZ, F_MZX, F_MYZ, F_MZY,  // momentum fluxes
  F_LX1, F_LX2, F_LY1, F_LY2, F_LZ1, F_LZ2,         // Lorentz products
  F_GX, F_GY, F_GZ, F_QT,                           // energy fluxes, -P div u + Q
  F_LFX, F_LFY, F_LFZ,                              // ln(rho/r0) interpolated to the faces
  F_LNX, F_LNY, F_LNZ,                              // ln<nu> interpolated to the faces
  F_SQXY, F_SQYZ, F_SQZX,                           // squared off-diagonal strain (edges)
  F_ED,                                             // e - e0 at centres
  F_LER,                                            // ln e - ln <e>_h (ediffav)
  F_LQ,                                             // ln(P / P_aver) (lnp_aver)
  F_COUNT
};

// Kernel identities for per-kernel timing.
enum KId { K_LR = 0, K_VEL, K_STRAIN2, K_NU_RAW, K_NU_MAX, K_NU_SMOOTH, K_NU_FACES, K_TAU, K_EDGE,
           K_FLUX, K_DIV, K_UPDATE, K_COURANT, K_DIAG, K_MISC, K_D2FLAG, K_COOL2, K_FLUX_E, K_NU_MS,
           K_FDIV, K_WALL, K_PLANE, K_COUNT };
extern const char* const KNAMES[K_COUNT];

struct Fused {
  Geo geo;
  KPar kp;
  float* fld[F_COUNT];
  float* q[8];          // dfdt (2N storage)
  float* ping[8];       // stage state buffers
  float* pong[8];
  double cdt, cdtr, cdtd, dlmin, dfac;  // Courant factors, dl_min, diffusion factor
  double* dt_dev;       // device step and the three limits
  float* bdt_dev;       // beta_s dt of the three RK stages, in FP32, written with dt_dev[0]
  double* red;          // reduction partials (diagnostics)
  unsigned* cmax;       // Courant maxima as float bits, cleared by each final pass
  unsigned char* d2flag;  // second-order switch flags per cell (bit = axis), or null
  int zs;               // stretched z mesh
  float* mesh;          // its dz/dk and inverses on the device (4 nz floats), or null
  double wsum_f;        // sum of the z-face weights of the diagnostics (n when uniform)
  double* plane;        // plane means (nz) then per-block parts (nz * plane_nb), or null
  int plane_nb;
  double* pplane;       // the same for E - E0 (ln(P/P_aver)), then its 3 nz floats of
                        // per-plane pressure factors, or null
  double* oplane;       // stellar-atmosphere means (zghost + 4), then their per-block parts
  float* pot;           // R27 scratch: roots (nx + ny), 6 complex and 2 real planes, or null
  int red_blocks;
  int cells4;           // nx % 4 == 0 and four-cell threads not switched off
  int fdiv;             // fluxes, divergences and update in one kernel (k_fdiv)
  int wall;             // closed z walls: ghost planes refilled before every stage
  long long launches;
  // Courant-mode step captured as a CUDA graph for the state arrays step_key
  // (step_state 0: not tried, 1: captured, -1: capture unavailable).
  int step_state;
  cudaGraphExec_t step_exec;
  cudaStream_t cap;
  float* step_key[8];
  long long step_launches;
  // Optional per-kernel timing with CUDA events on the launch stream.
  int timing;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  std::vector<cudaEvent_t> pool;
  double kt_ms[K_COUNT];
  long long kt_n[K_COUNT];
};

int fused_init(Fused& F, const stagger_grid& g, const stagger_params& p);
void fused_release(Fused& F);
// F(f) into out[8] (plain derivatives).
int fused_rhs(Fused& F, float* const f[8], float* out[8], cudaStream_t s);
// One RK3 step in place on f.  dt > 0 fixed, else Courant (device-side).
int fused_step(Fused& F, float* f[8], double dt, cudaStream_t s);
// The same step; a Courant-mode step (dt <= 0) with timing off replays a CUDA
// graph of its launches, captured once for these state arrays.
int fused_step_graphed(Fused& F, float* f[8], double dt, cudaStream_t s);
// The Courant step of state f and its three limits into F.dt_dev[0..3]
// (dt, t_wave, t_rate, t_diff), enqueued on s without synchronising.
int fused_dt(Fused& F, float* const f[8], cudaStream_t s);
// Courant limits (t_wave, t_rate, t_diff) and dt for state f, synchronising.
int fused_courant(Fused& F, float* const f[8], double lim[3], double* dt, cudaStream_t s);
// Per-kernel timing: on/off, and collect (synchronises the stream).
void fused_timing(Fused& F, int on);
int fused_collect(Fused& F, cudaStream_t s);
// FP64 diagnostics, synchronising.
int fused_diagnostics(Fused& F, float* const f[8], const stagger_params& p, double out[10],
                      cudaStream_t s);

}  // namespace stg
