// Fused FP32 forward path: one RK stage is eight launches, each a star
// stencil of reach <= 3 cells per axis over one or a few fields, with the
// intermediate fluxes kept in HBM between launches:
//   lr      ln(rho/r0)                                   (pointwise)
//   vel     u = p / rho_face                              (Sect. "Centering")
//   nu_raw  Richtmyer-Morton nu, eq. (RMnu)               (viscous runs)
//   nu_max  3x3x3 max;  nu_smooth  3x3x3 mean, ln<nu>      (Sect. "Richtmyer & Morton")
//   tau     stresses eq. (itv), eta J, J                  (edges, centres)
//   edge    quench eq. (quench), E = -u x B + eta J eq. (ohm), heating densities
//   flux    momentum, Lorentz and energy fluxes, -P div u + Q
//   div     divergences -> F(f), eqs. (mass) (mom) (ien) (indu), then the
//           low-storage update eqs. (ddt), (tupdate)
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "fused_kernels.cuh"
#include "stage_kernels.cuh"

namespace stg {

// ================================================================ host =====

const char* const KNAMES[K_COUNT] = {"k_lr_ed", "k_vel", "k_strain2", "k_nu_raw", "k_nu_max",
                                     "k_nu_smooth", "k_nu_faces", "k_tau", "k_edge", "k_flux",
                                     "k_div", "k_update", "k_courant", "k_diag", "k_misc",
                                     "k_d2flag", "k_cool2", "k_flux_e", "k_nu_maxsmooth",
                                     "k_fdiv", "k_wall", "k_plane"};

static cudaEvent_t ev_get(Fused& F) {
  if (!F.pool.empty()) {
    cudaEvent_t e = F.pool.back();
    F.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch bracket: count the launch and, when timing, record an event pair
// around it on the launch stream.
#define TIMED(kid, stmt)                                          \
  do {                                                            \
    cudaEvent_t e0_ = nullptr;                                    \
    if (F.timing) { e0_ = ev_get(F); cudaEventRecord(e0_, s); }   \
    stmt;                                                         \
    if (F.timing) {                                               \
      cudaEvent_t e1_ = ev_get(F);                                \
      cudaEventRecord(e1_, s);                                    \
      F.pending.push_back({(kid), {e0_, e1_}});                   \
    }                                                             \
    ++F.launches;                                                 \
  } while (0)

void fused_timing(Fused& F, int on) { F.timing = on; }

int fused_collect(Fused& F, cudaStream_t s) {
  STG_CUDA_OK(cudaStreamSynchronize(s));
  for (auto& pe : F.pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess) {
      F.kt_ms[pe.first] += ms;
      F.kt_n[pe.first] += 1;
    }
    F.pool.push_back(pe.second.first);
    F.pool.push_back(pe.second.second);
  }
  F.pending.clear();
  return STAGGER_OK;
}

static dim3 grid3(const Geo& g) {
  return dim3((unsigned)((g.nx + BX - 1) / BX), (unsigned)((g.ny + BY - 1) / BY),
              (unsigned)((g.nz + BZ - 1) / BZ));
}
static inline unsigned nb1(long long n) { return (unsigned)((n + 255) / 256); }

// Grid of the per-cell kernels for cell type N (N::W consecutive x-cells per thread).
template <class N> static dim3 grid_cells(const Geo& g) {
  return dim3((unsigned)((g.nx + BX * N::W - 1) / (BX * N::W)), (unsigned)((g.ny + BY - 1) / BY),
              (unsigned)((g.nz + BZ - 1) / BZ));
}

// Thread-block shapes of BX * BY * BZ threads, chosen per kernel by A/B runs
// on GB300 at 512^3: long in z (32 x 1 x 8) for k_tau, k_edge, k_flux and the
// divergences, long in y (32 x 8 x 1) for the energy fluxes, k_vel, k_nu_raw
// and k_nu_faces; the default 32 x 2 x 4 for the rest.
static_assert(BY * BZ == 8, "the per-kernel shapes keep the launch bounds' thread count");
static const dim3 BB_Z8(BX, 1, 8);
static const dim3 BB_Y8(BX, 8, 1);
template <class N> static dim3 grid_for(const Geo& g, dim3 b) {
  return dim3((unsigned)((g.nx + b.x * N::W - 1) / (b.x * N::W)), (unsigned)((g.ny + b.y - 1) / b.y),
              (unsigned)((g.nz + b.z - 1) / b.z));
}

// Four-cell threads need 16-byte aligned arrays (the workspace always is).
static bool aligned16(float* const* a, int n) {
  uintptr_t u = 0;
  for (int i = 0; i < n; ++i) u |= (uintptr_t)a[i];
  return (u & 15) == 0;
}

int fused_init(Fused& F, const stagger_grid& gr, const stagger_params& p) {
  F.geo = make_geo(gr.nx, gr.ny, gr.nz);
  F.step_state = 0;
  F.step_exec = nullptr;
  F.cap = nullptr;
  F.step_launches = 0;
  for (int c = 0; c < 8; ++c) F.step_key[c] = nullptr;
  F.cells4 = (gr.nx % 4) == 0 && !p.scalar_cells;
  // One z-marching flux-divergence kernel per stage (on request; uniform z only).
  F.fdiv = p.fuse_flux_div && p.zc == nullptr;
  // z walls at the planes zghost and nz - 1 - zghost: 0 periodic, 1 closed
  // (R22), 2 rigid (R25).
  F.wall = p.zwalls;
  F.launches = 0;
  F.timing = 0;
  for (int i = 0; i < K_COUNT; ++i) { F.kt_ms[i] = 0; F.kt_n[i] = 0; }

  KPar& k = F.kp;
  const double h[3] = {gr.dx, gr.dy, gr.dz};
  const int nn[3] = {gr.nx, gr.ny, gr.nz};
  // A stretched z (R19) takes its smallest and largest cell into the mesh's
  // dl_min and dl_max.
  const bool zs = p.zc != nullptr;
  double zcmin = 1e300, zcmax = 0, zcsum = 0, zfsum = 0;
  for (int kk = 0; zs && kk < gr.nz; ++kk) {
    zcmin = fmin(zcmin, p.zc[kk]);
    zcmax = fmax(zcmax, p.zc[kk]);
    zcsum += p.zc[kk];
    zfsum += p.zf[kk];
  }
  double dlmin = 1e300, dlxy = 1e300;
  int any = 0;
  for (int a = 0; a < 3; ++a)
    if (nn[a] > 1) {
      dlmin = fmin(dlmin, (a == 2 && zs) ? zcmin : h[a]);
      if (a < 2) dlxy = fmin(dlxy, h[a]);
      any = 1;
    }
  if (!any) dlmin = fmin(h[0], fmin(h[1], h[2]));
  double sp[3];
  for (int a = 0; a < 3; ++a) {
    k.ih[a] = (float)(1.0 / h[a]);
    sp[a] = nn[a] > 1 ? h[a] : dlmin;
    k.sp[a] = (float)sp[a];
  }
  k.spp[0] = (float)fmax(sp[1], sp[2]);
  k.spp[1] = (float)fmax(sp[2], sp[0]);
  k.spp[2] = (float)fmax(sp[0], sp[1]);
  k.r0 = (float)p.ref[0];
  k.E0 = (float)p.ref[4];
  k.r0pos = p.ref[0] > 0;
  k.e0 = p.ref[0] > 0 ? (float)(p.ref[4] / p.ref[0]) : 0.f;
  k.Ec = (float)(p.ref[4] - (double)k.e0 * p.ref[0]);
  for (int d = 0; d < 3; ++d) {
    k.pref[d] = (float)p.ref[1 + d];
    k.Bref[d] = (float)p.ref[5 + d];
    k.g[d] = (float)p.g[d];
  }
  k.gamma = (float)p.gamma;
  k.gm1 = (float)(p.gamma - 1.0);
  k.visc = (p.nu_const > 0 || p.nu1 > 0 || p.nu2 > 0 || p.nu3 > 0 || p.csmag > 0) ? 1 : 0;
  k.csmag_dl = (float)(p.csmag * dlmin);
  k.d2div = p.do_2nddiv && k.visc;
  k.d2lim = (float)p.d2lnr_lim;
  k.rm = k.visc && !(p.nu_const > 0);
  k.nu1 = (float)p.nu1;
  k.nu2dl = (float)(p.nu2 * dlmin);
  k.nu3 = (float)p.nu3;
  k.nu_const = (float)p.nu_const;
  k.nuE = (float)p.nuE;
  k.nuB = (float)p.nuB;
  k.c1 = (float)p.c1;
  k.inv_qmax = (float)(1.0 / p.qmax);
  k.qlim = (float)p.qlim;
  k.qmax3 = p.quench_max3 ? 1 : 0;
  k.qeps = (float)p.quench_eps;
  k.log_interp = p.log_interp ? 1 : 0;
  k.do_quench = p.do_quench ? 1 : 0;
  k.inv_tcool = p.t_cool > 0 ? (float)(1.0 / p.t_cool) : 0.f;
  k.e_cool = (float)p.e_cool;
  k.inv_rho_cool = p.cool_cut ? (float)(1.0 / p.rho_cool) : 0.f;
  k.cool_cut = p.cool_cut;
  double dlmax = 0;
  for (int a = 0; a < 3; ++a)
    if (nn[a] > 1 || !any) dlmax = fmax(dlmax, (a == 2 && zs) ? zcmax : h[a]);
  k.dlmin = (float)dlmin;
  k.dlxy = (float)fmin(dlxy, 1e30);
  k.nu2 = (float)p.nu2;
  k.csmag = (float)p.csmag;
  k.izbar = zs ? gr.nz / zcsum : 1.0;
  k.hzc = k.hzf = k.jzc = k.jzf = nullptr;
  k.inv_tchromo = p.t_chromo > 0 ? (float)(1.0 / p.t_chromo) : 0.f;
  k.inv_rhobot = p.t_chromo > 0 ? (float)(1.0 / p.rho_bot) : 0.f;
  k.emean = nullptr;
  k.corL0 = (float)p.cor_L0;
  k.corTu = (float)p.cor_Tunit;
  k.ediffav = p.ediffav && k.visc ? 1 : 0;
  k.lnpa = p.lnp_aver ? 1 : 0;
  k.Emean = nullptr;
  k.pa = k.paz = k.dpaz = k.qm = k.qden = nullptr;
  k.wall = p.zwalls;
  k.klo = p.zwalls ? p.zghost : 0;
  k.khi = p.zwalls ? gr.nz - 1 - p.zghost : gr.nz - 1;
  // Stellar-atmosphere boundaries (R26): the bottom is the end gravity points to.
  k.obot = p.g[2] < 0 ? k.klo : k.khi;
  k.otop = p.g[2] < 0 ? k.khi : k.klo;
  k.osb = p.g[2] < 0 ? -1 : 1;
  k.ost = -k.osb;
  k.oinv_t = (float)(1.0 / p.bdry_t);
  k.orho = (float)p.bdry_rho;
  k.oE = (float)p.bdry_E;
  k.oinv_u = (float)(1.0 / p.bdry_u);
  k.oBx = (float)p.bdry_B[0];
  k.oBy = (float)p.bdry_B[1];
  k.orlo = (float)p.top_rho_lo;
  k.orhi = (float)p.top_rho_hi;
  k.oefac = (float)p.top_e_fac;
  k.oumax = (float)p.top_umax;
  k.ogabs = (float)fabs(p.g[2]);
  k.omean = nullptr;
  k.oinv_tpot = (p.zwalls == 3 && p.top_tpot > 0) ? (float)(1.0 / p.top_tpot) : 0.f;
  k.bpx = k.bpy = nullptr;
  F.zs = zs ? 1 : 0;
  F.wsum_f = zs ? (double)gr.nx * gr.ny * zfsum * k.izbar : (double)F.geo.n;
  F.cdt = p.Cdt;
  F.cdtr = p.Cdtr;
  F.cdtd = p.Cdtd;
  F.dlmin = dlmin;
  F.dfac = fmax(1.0, fmax(p.nuE, p.nuB * dlmax / dlmin));

  const size_t bytes = sizeof(float) * (size_t)F.geo.n;
  for (int i = 0; i < F_COUNT; ++i) F.fld[i] = nullptr;
  for (int c = 0; c < 8; ++c) F.q[c] = F.ping[c] = F.pong[c] = nullptr;
  F.dt_dev = nullptr;
  F.bdt_dev = nullptr;
  F.red = nullptr;
  F.cmax = nullptr;
  F.d2flag = nullptr;
  F.mesh = nullptr;
  F.plane = nullptr;
  F.pplane = nullptr;
  F.oplane = nullptr;
  F.pot = nullptr;
  F.plane_nb = (int)std::max(1LL, std::min(64LL, ((long long)gr.nx * gr.ny + 1023) / 1024));
  if (k.lnpa) {
    // ln(P/P_aver): the plane means of E - E0 and their per-block parts, then
    // P_aver, exp(dn_z ln P_aver), dddn_z ln P_aver, <E'> and E0 + <E'> as 5 nz floats.
    const size_t nd = (size_t)gr.nz * (1 + F.plane_nb);
    if (cudaMalloc(&F.pplane, sizeof(double) * nd + sizeof(float) * 5 * (size_t)gr.nz) !=
        cudaSuccess) {
      F.pplane = nullptr;
      fused_release(F);
      return STAGGER_EOOM;
    }
    k.Emean = F.pplane;
    k.pa = reinterpret_cast<const float*>(F.pplane + nd);
    k.paz = k.pa + gr.nz;
    k.dpaz = k.pa + 2 * gr.nz;
    k.qm = k.pa + 3 * gr.nz;
    k.qden = k.pa + 4 * gr.nz;
  }
  if (F.wall == 3) {
    // Stellar-atmosphere boundaries: zghost + 2 plane means, then their parts.
    const size_t rows = (size_t)p.zghost + 4;
    if (cudaMalloc(&F.oplane, sizeof(double) * rows * (1 + F.plane_nb)) != cudaSuccess) {
      F.oplane = nullptr;
      fused_release(F);
      return STAGGER_EOOM;
    }
    k.omean = F.oplane;
  }
  if (k.oinv_tpot > 0.f) {
    // R27 scratch: the two target planes, the roots of unity along x and y,
    // and six complex planes of the transforms.
    const size_t m2 = (size_t)gr.nx * gr.ny;
    const size_t nfl = 14 * m2 + 2 * ((size_t)gr.nx + gr.ny);
    if (cudaMalloc(&F.pot, sizeof(float) * nfl) != cudaSuccess) {
      F.pot = nullptr;
      fused_release(F);
      return STAGGER_EOOM;
    }
    std::vector<float> w(2 * ((size_t)gr.nx + gr.ny));
    for (int r = 0; r < gr.nx; ++r) {
      w[2 * r] = (float)cos(2.0 * M_PI * r / gr.nx);
      w[2 * r + 1] = (float)-sin(2.0 * M_PI * r / gr.nx);
    }
    for (int r = 0; r < gr.ny; ++r) {
      w[2 * (gr.nx + r)] = (float)cos(2.0 * M_PI * r / gr.ny);
      w[2 * (gr.nx + r) + 1] = (float)-sin(2.0 * M_PI * r / gr.ny);
    }
    if (cudaMemcpy(F.pot + 2 * m2, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      fused_release(F);
      return STAGGER_ECUDA;
    }
    k.bpx = F.pot;
    k.bpy = F.pot + m2;
    // The row transforms keep the nx roots in shared memory.
    const int sm = (int)(sizeof(float2) * (size_t)gr.nx);
    if (sm > 48 * 1024 &&
        (cudaFuncSetAttribute(k_dft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) !=
             cudaSuccess ||
         cudaFuncSetAttribute(k_idft_rows2, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) !=
             cudaSuccess)) {
      fused_release(F);
      return STAGGER_ECUDA;
    }
  }
  if (p.t_chromo > 0 || k.ediffav) {
    // Plane means of e for the chromospheric cooling and the energy diffusion
    // of eq. (ediffav): nz means, then the per-block parts of the fixed-order
    // reduction.
    if (cudaMalloc(&F.plane, sizeof(double) * (size_t)gr.nz * (1 + F.plane_nb)) != cudaSuccess) {
      F.plane = nullptr;
      fused_release(F);
      return STAGGER_EOOM;
    }
    k.emean = F.plane;
  }
  if (zs) {
    // dz/dk at centres and faces and their inverses, as four arrays of nz.
    std::vector<float> m((size_t)4 * gr.nz);
    for (int kk = 0; kk < gr.nz; ++kk) {
      m[kk] = (float)p.zc[kk];
      m[gr.nz + kk] = (float)p.zf[kk];
      m[2 * gr.nz + kk] = (float)(1.0 / p.zc[kk]);
      m[3 * gr.nz + kk] = (float)(1.0 / p.zf[kk]);
    }
    if (cudaMalloc(&F.mesh, sizeof(float) * m.size()) != cudaSuccess) {
      F.mesh = nullptr;
      fused_release(F);
      return STAGGER_EOOM;
    }
    if (cudaMemcpy(F.mesh, m.data(), sizeof(float) * m.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      fused_release(F);
      return STAGGER_ECUDA;
    }
    k.hzc = F.mesh;
    k.hzf = F.mesh + gr.nz;
    k.jzc = F.mesh + 2 * gr.nz;
    k.jzf = F.mesh + 3 * gr.nz;
  }
  // Which intermediate fields this parameter set needs.
  std::vector<int> need = {F_UX, F_UY, F_UZ};
  // The fused flux-divergence kernel keeps every flux on chip and forms J
  // itself; k_tau still writes J and eta J for k_edge in viscous runs.
  if (!F.fdiv || k.visc) for (int f : {F_JX, F_JY, F_JZ, F_EX, F_EY, F_EZ}) need.push_back(f);
  if (!F.fdiv)
    for (int f : {F_MXX, F_MYY, F_MZZ, F_MXY, F_MYX, F_MXZ, F_MZX, F_MYZ, F_MZY, F_LX1, F_LX2,
                  F_LY1, F_LY2, F_LZ1, F_LZ2, F_GX, F_GY, F_GZ, F_QT})
      need.push_back(f);
  need.push_back(F_ED);
  if (k.ediffav) need.push_back(F_LER);
  if (k.lnpa) need.push_back(F_LQ);
  if (k.log_interp) need.push_back(F_LR);
  if (k.rm) for (int f : {F_NV, F_NM, F_NU, F_LNU, F_LNX, F_LNY, F_LNZ}) need.push_back(f);
  if (k.csmag_dl > 0.f) for (int f : {F_SQXY, F_SQYZ, F_SQZX}) need.push_back(f);
  if (k.visc)
    for (int f : {F_TXX, F_TYY, F_TZZ, F_TXY, F_TYZ, F_TZX, F_RX, F_RY, F_RZ, F_WC, F_WX, F_WY, F_WZ,
                  F_LFX, F_LFY, F_LFZ})
      need.push_back(f);
  if (k.visc && k.do_quench)
    for (int f : {F_QXX, F_QYY, F_QZZ, F_QXY, F_QYZ, F_QZX}) need.push_back(f);
  for (int f : need)
    if (cudaMalloc(&F.fld[f], bytes) != cudaSuccess) { F.fld[f] = nullptr; fused_release(F); return STAGGER_EOOM; }
  for (int c = 0; c < 8; ++c) {
    if (cudaMalloc(&F.q[c], bytes) != cudaSuccess || cudaMalloc(&F.ping[c], bytes) != cudaSuccess ||
        cudaMalloc(&F.pong[c], bytes) != cudaSuccess) {
      fused_release(F);
      return STAGGER_EOOM;
    }
  }
  dim3 gg = grid3(F.geo);
  F.red_blocks = (int)(gg.x * gg.y * gg.z);
  if (k.d2div && cudaMalloc(&F.d2flag, (size_t)F.geo.n) != cudaSuccess) {
    F.d2flag = nullptr;
    fused_release(F);
    return STAGGER_EOOM;
  }
  if (cudaMalloc(&F.cmax, sizeof(unsigned) * 4) != cudaSuccess ||
      cudaMemset(F.cmax, 0, sizeof(unsigned) * 4) != cudaSuccess) {
    fused_release(F);
    return STAGGER_EOOM;
  }
  if (cudaMalloc(&F.dt_dev, sizeof(double) * 8) != cudaSuccess ||
      cudaMalloc(&F.bdt_dev, sizeof(float) * 4) != cudaSuccess ||
      cudaMalloc(&F.red, sizeof(double) * 10 * (size_t)F.red_blocks) != cudaSuccess) {
    fused_release(F);
    return STAGGER_EOOM;
  }
  return STAGGER_OK;
}

void fused_release(Fused& F) {
  if (F.step_exec) cudaGraphExecDestroy(F.step_exec);
  F.step_exec = nullptr;
  if (F.cap) cudaStreamDestroy(F.cap);
  F.cap = nullptr;
  for (auto& pe : F.pending) { cudaEventDestroy(pe.second.first); cudaEventDestroy(pe.second.second); }
  F.pending.clear();
  for (auto e : F.pool) cudaEventDestroy(e);
  F.pool.clear();
  for (int i = 0; i < F_COUNT; ++i) { if (F.fld[i]) cudaFree(F.fld[i]); F.fld[i] = nullptr; }
  for (int c = 0; c < 8; ++c) {
    if (F.q[c]) cudaFree(F.q[c]);
    if (F.ping[c]) cudaFree(F.ping[c]);
    if (F.pong[c]) cudaFree(F.pong[c]);
    F.q[c] = F.ping[c] = F.pong[c] = nullptr;
  }
  if (F.dt_dev) cudaFree(F.dt_dev);
  if (F.bdt_dev) cudaFree(F.bdt_dev);
  if (F.red) cudaFree(F.red);
  if (F.cmax) cudaFree(F.cmax);
  F.cmax = nullptr;
  if (F.d2flag) cudaFree(F.d2flag);
  F.d2flag = nullptr;
  if (F.mesh) cudaFree(F.mesh);
  F.mesh = nullptr;
  if (F.plane) cudaFree(F.plane);
  F.plane = nullptr;
  if (F.pplane) cudaFree(F.pplane);
  F.pplane = nullptr;
  if (F.oplane) cudaFree(F.oplane);
  F.oplane = nullptr;
  if (F.pot) cudaFree(F.pot);
  F.pot = nullptr;
  F.dt_dev = nullptr;
  F.bdt_dev = nullptr;
  F.red = nullptr;
}

// Everything up to (not including) the divergence kernel: primitives,
// viscosity, stresses, edge fields and fluxes of state f.
template <class N>
static int pre_div_t(Fused& F, float* const f[8], cudaStream_t s, bool cfl) {
  const Geo& g = F.geo;
  const KPar& k = F.kp;
  float** d = F.fld;
  const dim3 gg = grid_cells<N>(g), bb(BX, BY, BZ);
  const dim3 gz8 = grid_for<N>(g, BB_Z8), gy8 = grid_for<N>(g, BB_Y8);
  using NB = typename N::Base;   // kernels without derivatives or lengths
  const float* ls = k.log_interp ? d[F_LR] : f[0];
  // Plane means of e - e0 (chromospheric cooling, eq. (ediffav)), before the
  // kernels that read them.
  if (k.inv_tchromo > 0.f || k.ediffav) {
    TIMED(K_PLANE, (k_plane_part<false><<<dim3(F.plane_nb, g.nz), 256, 0, s>>>(
                       f[0], f[4], F.plane + g.nz, k, g)));
    TIMED(K_PLANE, (k_plane_final<<<(g.nz + 63) / 64, 64, 0, s>>>(F.plane + g.nz, F.plane_nb,
                                                                   F.plane, g)));
  }
  if (k.lnpa) {   // ln(P/P_aver), eq. (pressure): plane means of E - E0, P_aver factors
    TIMED(K_PLANE, (k_plane_part<true><<<dim3(F.plane_nb, g.nz), 256, 0, s>>>(
                       f[0], f[4], F.pplane + g.nz, k, g)));
    TIMED(K_PLANE, (k_lnpa_tab<<<1, 256, 0, s>>>(F.pplane + g.nz, F.plane_nb, F.pplane,
                                                 const_cast<float*>(k.pa),
                                                 const_cast<float*>(k.paz),
                                                 const_cast<float*>(k.dpaz),
                                                 const_cast<float*>(k.qm),
                                                 const_cast<float*>(k.qden), k, g)));
  }
  TIMED(K_LR, (k_lr_ed<NB><<<nb1(g.n / N::W), 256, 0, s>>>(f[0], f[4], k.log_interp ? d[F_LR] : nullptr,
                                                       d[F_ED], k.ediffav ? d[F_LER] : nullptr,
                                                       k.lnpa ? d[F_LQ] : nullptr, k, g.n, g.sz)));
  TIMED(K_VEL, (k_vel<NB><<<gy8, BB_Y8, 0, s>>>(ls, f[1], f[2], f[3], d[F_UX], d[F_UY], d[F_UZ],
                                        d[F_LFX], d[F_LFY], d[F_LFZ], k, g)));
  if (k.rm) {
    if (k.csmag_dl > 0.f)
      TIMED(K_STRAIN2, (k_strain2<N><<<gg, bb, 0, s>>>(d[F_UX], d[F_UY], d[F_UZ], d[F_SQXY], d[F_SQYZ],
                                                    d[F_SQZX], k, g)));
    // cfl: this stage's derivative sets the Courant step, and the wave-speed
    // and <nu> maxima are taken here (cmax[0], cmax[2]).
    auto knu = k.csmag_dl > 0.f ? (cfl ? k_nu_raw<true, true, N> : k_nu_raw<true, false, N>)
                                : (cfl ? k_nu_raw<false, true, N> : k_nu_raw<false, false, N>);
    TIMED(K_NU_RAW, (knu<<<gy8, BB_Y8, 0, s>>>(d[F_UX], d[F_UY], d[F_UZ], f[0], f[4], f[5], f[6], f[7],
                                           d[F_SQXY], d[F_SQYZ], d[F_SQZX], d[F_NV],
                                           cfl ? F.cmax : nullptr, k, g)));
    if (N::W == 4) {
      // One z-marching pass for the 3x3x3 max and mean (four-cell layout).
      const dim3 gm((unsigned)((g.nx + 127) / 128), (unsigned)((g.ny + NUZ_TY - 1) / NUZ_TY),
                    (unsigned)((g.nz + NUZ_ZC - 1) / NUZ_ZC));
      auto kms = cfl ? k_nu_maxsmooth<true> : k_nu_maxsmooth<false>;
      TIMED(K_NU_MS, (kms<<<gm, dim3(32, NUZ_TY), 0, s>>>(d[F_NV], d[F_NU], d[F_LNU], F.cmax + 2, g)));
    } else {
      TIMED(K_NU_MAX, (k_nu_max<NB><<<gg, bb, 0, s>>>(d[F_NV], d[F_NM], g)));
      auto ksm = cfl ? k_nu_smooth<NB, true> : k_nu_smooth<NB, false>;
      TIMED(K_NU_SMOOTH, (ksm<<<gg, bb, 0, s>>>(d[F_NM], d[F_NU], d[F_LNU], F.cmax + 2, g)));
    }
    TIMED(K_NU_FACES, (k_nu_faces<NB><<<gy8, BB_Y8, 0, s>>>(d[F_LNU], d[F_LNX], d[F_LNY], d[F_LNZ], g)));
  }
  if (k.d2div)
    TIMED(K_D2FLAG, (k_d2flag<NB><<<gg, bb, 0, s>>>(f[0], f[4], F.d2flag, k, g)));
  // The fused flux-divergence kernel forms J itself: k_tau only for viscous runs.
  auto ktau = k.d2div ? k_tau<N, true> : k_tau<N, false>;
  if (!F.fdiv || k.visc)
  TIMED(K_TAU, (ktau<<<gz8, BB_Z8, 0, s>>>(d[F_UX], d[F_UY], d[F_UZ], f[0], d[F_LFX], d[F_LFY],
                                       d[F_LFZ], d[F_NU], d[F_LNX], d[F_LNY], d[F_LNZ], f[5],
                                       f[6], f[7], d[F_TXX], d[F_TYY], d[F_TZZ], d[F_TXY],
                                       d[F_TYZ], d[F_TZX], d[F_RX], d[F_RY], d[F_RZ], d[F_JX],
                                       d[F_JY], d[F_JZ], F.d2flag, k, g)));
  auto kedge = k.qmax3 ? (k.d2div ? k_edge<N, true, true> : k_edge<N, false, true>)
                       : (k.d2div ? k_edge<N, true, false> : k_edge<N, false, false>);
  if (k.visc)
    TIMED(K_EDGE, (kedge<<<gz8, BB_Z8, 0, s>>>(d[F_TXX], d[F_TYY], d[F_TZZ], d[F_TXY], d[F_TYZ],
                                           d[F_TZX], d[F_RX], d[F_RY], d[F_RZ], d[F_JX],
                                           d[F_JY], d[F_JZ], d[F_UX], d[F_UY], d[F_UZ],
                                           d[F_QXX], d[F_QYY], d[F_QZZ], d[F_QXY], d[F_QYZ],
                                           d[F_QZX], d[F_EX], d[F_EY], d[F_EZ], d[F_WC],
                                           d[F_WX], d[F_WY], d[F_WZ], F.d2flag, k, g)));
  if (F.fdiv) {   // fluxes, divergences and update in k_fdiv (launch_div)
    STG_CUDA_OK(cudaGetLastError());
    return STAGGER_OK;
  }
  const bool qn = k.visc && k.do_quench;
  FluxIn fi = {f[1], f[2], f[3], f[0], f[4], f[5], f[6], f[7], ls, d[F_UX], d[F_UY], d[F_UZ],
               qn ? d[F_QXX] : d[F_TXX], qn ? d[F_QYY] : d[F_TYY], qn ? d[F_QZZ] : d[F_TZZ],
               qn ? d[F_QXY] : d[F_TXY], qn ? d[F_QYZ] : d[F_TYZ], qn ? d[F_QZX] : d[F_TZX],
               d[F_JX], d[F_JY], d[F_JZ], d[F_NU], d[F_WC], d[F_WX], d[F_WY], d[F_WZ],
               d[F_ED], d[F_LER]};
  FluxOut fo = {d[F_MXX], d[F_MYY], d[F_MZZ], d[F_MXY], d[F_MYX], d[F_MXZ], d[F_MZX],
                d[F_MYZ], d[F_MZY], d[F_LX1], d[F_LX2], d[F_LY1], d[F_LY2], d[F_LZ1],
                d[F_LZ2], d[F_GX], d[F_GY], d[F_GZ], d[F_QT], d[F_EX], d[F_EY], d[F_EZ]};
  TIMED(K_FLUX, (k_flux<N><<<gz8, BB_Z8, 0, s>>>(fi, fo, k, g)));
  TIMED(K_FLUX_E, (k_flux_e<N><<<gy8, BB_Y8, 0, s>>>(fi, fo, k, g)));
  if (k.inv_tchromo > 0.f || k.corL0 > 0.f)
    TIMED(K_COOL2, (k_cool2<NB><<<gg, bb, 0, s>>>(f[0], f[4], d[F_QT], k, g)));
  STG_CUDA_OK(cudaGetLastError());
  return STAGGER_OK;
}

// The Courant maxima are taken inside the stage kernels (wave speed in
// k_nu_raw, <nu> in k_nu_maxsmooth or k_nu_smooth, rate in the mass and energy
// k_div) when RM viscosity runs on a uniform mesh; otherwise by k_courant_part.
static bool cfl_fused(const Fused& F) { return F.kp.rm && !F.zs && !F.wall; }

// Closed z walls: fill the ghost planes of the eight state arrays f (and
// zero the odd centred fields on the boundary planes), or zero the ghost
// planes of a time derivative.  Rigid z walls: the ghost momenta of f.
// ln(rho/r0) of the planes the ghost-momentum fills read (with log
// interpolation): 0..klo+3 and khi-3..nz-1, into F_LR, after the density of the
// ghost planes is final.  Returns F_LR, or null without log interpolation.
static const float* wall_lr(Fused& F, float* const f[8], cudaStream_t s) {
  const KPar& k = F.kp;
  const Geo& g = F.geo;
  if (!k.log_interp) return nullptr;
  float** d = F.fld;
  const int lo = std::min(k.klo + 4, g.nz), hi0 = std::max(k.khi - 3, lo);
  const long long r[2][2] = {{0, lo}, {hi0, g.nz}};
  for (int i = 0; i < 2; ++i) {
    const long long off = r[i][0] * g.sz, n = (r[i][1] - r[i][0]) * g.sz;
    if (n <= 0) continue;
    TIMED(K_WALL, (k_lr_ed<Nb><<<nb1(n), 256, 0, s>>>(f[0] + off, f[4] + off, d[F_LR] + off,
                                                       d[F_ED] + off, nullptr, nullptr, k, n,
                                                       g.sz)));
  }
  return d[F_LR];
}

// rhs: a right-hand side of f follows (the R27 targets are formed only then).
static void wall_launch(Fused& F, float* const f[8], bool zero, cudaStream_t s, bool rhs = true) {
  const Geo& g = F.geo;
  if (F.wall == 3) {
    // Stellar-atmosphere boundaries (R26): the divergence kernels write zero
    // derivatives on the ghost planes; a state gets its ghost planes from the
    // plane means, the rho and E extrapolation, then momenta and field.
    if (zero) return;
    const KPar& k = F.kp;
    const int G = k.klo, rows = G + 4;
    TIMED(K_WALL, (k_open_part<<<dim3(F.plane_nb, rows), 256, 0, s>>>(
                      f[0], f[1], f[2], f[5], f[6], F.oplane + rows, k, g)));
    TIMED(K_WALL, (k_open_final<<<(rows + 63) / 64, 64, 0, s>>>(F.oplane + rows, F.plane_nb,
                                                                  rows, F.oplane, g)));
    const unsigned bx = (unsigned)((g.sz + 255) / 256);
    TIMED(K_WALL, (k_open_fill_c<<<dim3(bx, 2 * G), 256, 0, s>>>(f[0], f[4], k, g)));
    const float* lr = wall_lr(F, f, s);
    TIMED(K_WALL, (k_open_fill_m<<<dim3(bx, 2 * G + 1), 256, 0, s>>>(f[1], f[2], f[3], f[5],
                                                                      f[6], f[7], f[0], lr, k, g)));
    if (k.oinv_tpot > 0.f && rhs) {
      // R27: the potential-field targets of the top plane from B_z on its
      // inside face, by horizontal Fourier modes.
      const int nx = g.nx, ny = g.ny;
      const size_t m2 = (size_t)nx * ny;
      float* bpx = F.pot;
      float* bpy = F.pot + m2;
      const float2* wx = reinterpret_cast<const float2*>(F.pot + 2 * m2);
      const float2* wy = wx + nx;
      float2* X = reinterpret_cast<float2*>(F.pot + 2 * m2 + 2 * ((size_t)nx + ny));
      float2 *Y = X + m2, *Px = Y + m2, *Py = Px + m2, *Zx = Py + m2, *Zy = Zx + m2;
      const int mi = k.ost > 0 ? k.khi : k.klo + 1;
      const dim3 gp((unsigned)((nx + 127) / 128), (unsigned)ny);
      const float Lx = (float)(nx / (double)k.ih[0]), Ly = (float)(ny / (double)k.ih[1]);
      const size_t sm = sizeof(float2) * (size_t)nx;   // the x roots in shared memory
      TIMED(K_WALL, (k_dft_rows<<<gp, 128, sm, s>>>(f[7] + (long long)mi * g.sz, X, wx, nx, ny)));
      TIMED(K_WALL, (k_dft_cols<<<gp, 128, 0, s>>>(X, Y, wy, nx, ny)));
      TIMED(K_WALL, (k_pot_sym<<<gp, 128, 0, s>>>(Y, Px, Py, nx, ny, Lx, Ly, (float)k.ost)));
      TIMED(K_WALL, (k_idft_cols2<<<gp, 128, 0, s>>>(Px, Py, Zx, Zy, wy, nx, ny)));
      TIMED(K_WALL, (k_idft_rows2<<<gp, 128, sm, s>>>(Zx, Zy, bpx, bpy, wx, nx, ny)));
    }
    return;
  }
  if (F.wall == 2) {
    // Rigid walls: the divergence kernels write zero derivatives on the ghost
    // planes; a state gets the ghost momenta of its boundary velocity.
    if (zero) return;
    Mom3 m = {{f[1], f[2], f[3]}};
    const int lb = F.kp.klo, ub = F.kp.khi;
    const dim3 gr((unsigned)((g.sz + 255) / 256), (unsigned)(lb + (g.nz - 1 - ub)), 3);
    const float* lr = wall_lr(F, f, s);
    TIMED(K_WALL, (k_rigid_fill<<<gr, 256, 0, s>>>(m, f[0], lr, F.kp, lb, ub, g)));
    return;
  }
  Wall8 w;
  for (int c = 0; c < 8; ++c) w.f[c] = f[c];
  const int lb = F.kp.klo, ub = F.kp.khi;
  const dim3 gg((unsigned)((g.sz + 255) / 256), (unsigned)(lb + 1 + (g.nz - ub)), 8);
  if (zero)
    TIMED(K_WALL, (k_wall_zero<<<gg, 256, 0, s>>>(w, lb, ub, g)));
  else
    TIMED(K_WALL, (k_wall_fill<<<gg, 256, 0, s>>>(w, lb, ub, g)));
}

static int pre_div(Fused& F, float* const f[8], cudaStream_t s, bool cfl = false) {
  const bool v4 = F.cells4 && aligned16(f, 8);
  if (F.zs) return v4 ? pre_div_t<Nb4Z>(F, f, s, false) : pre_div_t<NbZ>(F, f, s, false);
  return v4 ? pre_div_t<Nb4>(F, f, s, cfl) : pre_div_t<Nb>(F, f, s, cfl);
}

static DivIn div_in(Fused& F, float* const f[8]) {
  float** d = F.fld;
  DivIn di;
  di.px = f[1]; di.py = f[2]; di.pz = f[3];
  di.mxx = d[F_MXX]; di.myy = d[F_MYY]; di.mzz = d[F_MZZ]; di.mxy = d[F_MXY]; di.myx = d[F_MYX];
  di.mxz = d[F_MXZ]; di.mzx = d[F_MZX]; di.myz = d[F_MYZ]; di.mzy = d[F_MZY];
  di.lx1 = d[F_LX1]; di.lx2 = d[F_LX2]; di.ly1 = d[F_LY1]; di.ly2 = d[F_LY2];
  di.lz1 = d[F_LZ1]; di.lz2 = d[F_LZ2];
  di.gx = d[F_GX]; di.gy = d[F_GY]; di.gz = d[F_GZ]; di.qt = d[F_QT];
  di.Ex = d[F_EX]; di.Ey = d[F_EY]; di.Ez = d[F_EZ];
  di.ls = F.kp.log_interp ? d[F_LR] : f[0];
  for (int c = 0; c < 8; ++c) di.f[c] = f[c];
  di.lq = d[F_LQ];
  di.uz = d[F_UZ];
  return di;
}

// Stage inputs of k_fdiv: the state, the primitives of k_lr_ed and k_vel, and
// the viscous fields of k_tau, k_nu_* and k_edge.
static FdIn fdiv_in(Fused& F, float* const f[8]) {
  float** d = F.fld;
  const KPar& k = F.kp;
  const bool qn = k.visc && k.do_quench;
  FdIn in;
  for (int c = 0; c < 8; ++c) in.f[c] = f[c];
  in.ux = d[F_UX]; in.uy = d[F_UY]; in.uz = d[F_UZ];
  in.ed = d[F_ED];
  in.ler = d[F_LER];
  in.ls = k.log_interp ? d[F_LR] : f[0];
  in.txx = qn ? d[F_QXX] : d[F_TXX]; in.tyy = qn ? d[F_QYY] : d[F_TYY];
  in.tzz = qn ? d[F_QZZ] : d[F_TZZ]; in.txy = qn ? d[F_QXY] : d[F_TXY];
  in.tyz = qn ? d[F_QYZ] : d[F_TYZ]; in.tzx = qn ? d[F_QZX] : d[F_TZX];
  in.rx = d[F_EX]; in.ry = d[F_EY]; in.rz = d[F_EZ];   // eta J left by k_edge
  in.nu = d[F_NU];
  in.wc = d[F_WC]; in.wx = d[F_WX]; in.wy = d[F_WY]; in.wz = d[F_WZ];
  return in;
}

#ifndef FD_TY
#define FD_TY 8
#endif

static int launch_fdiv(Fused& F, float* const f[8], float* q[8], float* const* oo, float alpha,
                       int stg, int mode, cudaStream_t s, bool cfl) {
  const Geo& g = F.geo;
  const FdIn in = fdiv_in(F, f);
  const dim3 bb(FD_TX, FD_TY),
      gg((unsigned)((g.nx + FD_TX - 1) / FD_TX), (unsigned)((g.ny + FD_TY - 1) / FD_TY),
         (unsigned)((g.nz + FD_ZC - 1) / FD_ZC));
  typedef void (*FdK)(FdIn, float*, float*, float*, float*, float*, float*, float*, float*,
                      float*, float*, float*, float*, float*, float*, float*, float*, float,
                      const float*, int, unsigned*, KPar, Geo);
  FdK kern;
  if (F.kp.visc)
    kern = cfl ? k_fdiv<FD_TY, true, true> : k_fdiv<FD_TY, true, false>;
  else
    kern = cfl ? k_fdiv<FD_TY, false, true> : k_fdiv<FD_TY, false, false>;
  const size_t smem = fd_smem_bytes(FD_TY);
  if (smem > 48 * 1024)
    STG_CUDA_OK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  TIMED(K_FDIV, (kern<<<gg, bb, smem, s>>>(in, q[0], q[1], q[2], q[3], q[4], q[5], q[6], q[7],
                                        oo[0], oo[1], oo[2], oo[3], oo[4], oo[5], oo[6], oo[7],
                                        alpha, F.bdt_dev + stg, mode, F.cmax + 1, F.kp, g)));
  STG_CUDA_OK(cudaGetLastError());
  return STAGGER_OK;
}

// Stage stg's right-hand side into q (mode 0), or with the update by its
// beta dt (mode 1: F.bdt_dev[stg]).
static int launch_div(Fused& F, float* const f[8], float* q[8], float* o[8], float alpha,
                      int stg, int mode, cudaStream_t s, bool cfl = false) {
  if (F.fdiv) {
    float* oo[8];
    for (int c = 0; c < 8; ++c) oo[c] = o ? o[c] : q[c];
    return launch_fdiv(F, f, q, oo, alpha, stg, mode, s, cfl);
  }
  DivIn di = div_in(F, f);
  float* oo[8];
  for (int c = 0; c < 8; ++c) oo[c] = o ? o[c] : q[c];
  const bool v4 = F.cells4 && aligned16(f, 8) && aligned16(q, 8) && aligned16(oo, 8);
  const dim3 bb = BB_Z8, gg = v4 ? grid_for<Nb4>(F.geo, bb) : grid_for<Nb>(F.geo, bb);
  // Momentum; mass and energy; induction (disjoint inputs, one kernel each).
  const int nk = 3;
  typedef void (*DivK)(DivIn, float*, float*, float*, float*, float*, float*, float*, float*,
                       float*, float*, float*, float*, float*, float*, float*, float*, float,
                       const float*, int, unsigned*, KPar, Geo);
  DivK kern[3];
  if (F.zs) {
    kern[0] = v4 ? k_div<Nb4Z, 0x0E, false> : k_div<NbZ, 0x0E, false>;
    kern[1] = v4 ? k_div<Nb4Z, 0x11, false> : k_div<NbZ, 0x11, false>;
    kern[2] = v4 ? k_div<Nb4Z, 0xE0, false> : k_div<NbZ, 0xE0, false>;
  } else {
    if (F.wall >= 2) {   // rigid or stellar-atmosphere walls: the boundary branches
      kern[0] = v4 ? k_div<Nb4, 0x0E, false, true> : k_div<Nb, 0x0E, false, true>;
      kern[1] = v4 ? k_div<Nb4, 0x11, false, true> : k_div<Nb, 0x11, false, true>;
      kern[2] = v4 ? k_div<Nb4, 0xE0, false, true> : k_div<Nb, 0xE0, false, true>;
    } else {
      kern[0] = v4 ? k_div<Nb4, 0x0E, false> : k_div<Nb, 0x0E, false>;
      if (cfl)   // and the rate maximum (cmax[1])
        kern[1] = v4 ? k_div<Nb4, 0x11, true> : k_div<Nb, 0x11, true>;
      else
        kern[1] = v4 ? k_div<Nb4, 0x11, false> : k_div<Nb, 0x11, false>;
      kern[2] = v4 ? k_div<Nb4, 0xE0, false> : k_div<Nb, 0xE0, false>;
    }
  }
  for (int i = 0; i < nk; ++i)
    TIMED(K_DIV, (kern[i]<<<gg, bb, 0, s>>>(di, q[0], q[1], q[2], q[3], q[4], q[5], q[6], q[7],
                                            oo[0], oo[1], oo[2], oo[3], oo[4], oo[5], oo[6],
                                            oo[7], alpha, F.bdt_dev + stg, mode, F.cmax + 1,
                                            F.kp, F.geo)));
  STG_CUDA_OK(cudaGetLastError());
  return STAGGER_OK;
}

int fused_rhs(Fused& F, float* const f[8], float* out[8], cudaStream_t s) {
  if (F.wall) wall_launch(F, f, false, s);
  int st = pre_div(F, f, s);
  if (st) return st;
  st = launch_div(F, f, out, nullptr, 0.f, 0, 0, s);
  if (st) return st;
  if (F.wall) wall_launch(F, out, true, s);
  STG_CUDA_OK(cudaGetLastError());
  return STAGGER_OK;
}

template <class N>
static void courant_part(Fused& F, float* const f[8], cudaStream_t s) {
  TIMED(K_COURANT, (k_courant_part<N><<<grid_cells<N>(F.geo), dim3(BX, BY, BZ), 0, s>>>(
                       F.fld[F_UX], F.fld[F_UY], F.fld[F_UZ], f[0], f[4], f[5], f[6], f[7],
                       F.q[0], F.q[4], F.fld[F_NU], F.cmax, F.kp, F.geo)));
}

static int courant_to_dev(Fused& F, float* const f[8], cudaStream_t s, bool fused) {
  // Uses the primitives and <nu> that pre_div left for this state and q = F(f);
  // with fused, the stage kernels already took the three maxima.
  const bool v4 = F.cells4 && aligned16(f, 8);
  if (fused) {
  } else if (F.zs) {
    if (v4) courant_part<Nb4Z>(F, f, s); else courant_part<NbZ>(F, f, s);
  } else {
    if (v4) courant_part<Nb4>(F, f, s); else courant_part<Nb>(F, f, s);
  }
  // A stretched z reduces w / dl and nu / dl per cell: the final pass then
  // takes dl = 1 and a velocity-like nu.
  TIMED(K_COURANT, (k_courant_final<<<1, 32, 0, s>>>(
                        F.cmax, F.dt_dev, F.bdt_dev, (float)RK_BETA[0], (float)RK_BETA[1],
                        (float)RK_BETA[2], F.cdt, F.cdtr, F.cdtd, F.zs ? 1.0 : F.dlmin, F.dfac,
                        F.zs ? 1 : F.kp.rm)));
  return STAGGER_OK;
}

int fused_step(Fused& F, float* f[8], double dt, cudaStream_t s) {
  float* A[8];
  float* B[8];
  float* C[8];
  for (int c = 0; c < 8; ++c) { A[c] = f[c]; B[c] = F.ping[c]; C[c] = F.pong[c]; }
  float* const* st_in[3] = {A, B, C};
  float* const* st_out[3] = {B, C, A};
  for (int stg = 0; stg < 3; ++stg) {
    const bool cfl = stg == 0 && dt <= 0 && cfl_fused(F);
    // z walls: the stage input's ghost planes from its physical planes.
    if (F.wall) wall_launch(F, st_in[stg], false, s);
    int rc = pre_div(F, st_in[stg], s, cfl);
    if (rc) return rc;
    const float alpha = (float)RK_ALPHA[stg];
    if (stg == 0 && dt <= 0) {
      // Courant step from the state and its stage-1 derivative, then update.
      rc = launch_div(F, st_in[0], F.q, nullptr, 0.f, 0, 0, s, cfl);
      if (rc) return rc;
      courant_to_dev(F, st_in[0], s, cfl);
      Upd8 u;
      int vec = (F.geo.n % 4) == 0;
      for (int c = 0; c < 8; ++c) {
        u.f[c] = st_in[0][c];
        u.q[c] = F.q[c];
        u.o[c] = st_out[0][c];
        vec &= (((uintptr_t)u.f[c] | (uintptr_t)u.q[c] | (uintptr_t)u.o[c]) & 15) == 0;
      }
      const long long work = vec ? F.geo.n / 4 : F.geo.n;
      unsigned bx = (unsigned)((work + 255) / 256);
      if (bx > 2048) bx = 2048;
      TIMED(K_UPDATE, (k_update8<<<dim3(bx, 8), 256, 0, s>>>(u, F.bdt_dev, F.geo.n, vec)));
      STG_CUDA_OK(cudaGetLastError());
      continue;
    }
    if (stg == 0 && dt > 0) {
      TIMED(K_MISC, (k_set_dt<<<1, 1, 0, s>>>(F.dt_dev, F.bdt_dev, dt, (float)RK_BETA[0],
                                              (float)RK_BETA[1], (float)RK_BETA[2])));
    }
    rc = launch_div(F, st_in[stg], F.q, const_cast<float**>(st_out[stg]), alpha, stg, 1, s);
    if (rc) return rc;
  }
  if (F.wall) wall_launch(F, f, false, s, false);
  STG_CUDA_OK(cudaGetLastError());
  return STAGGER_OK;
}

int fused_dt(Fused& F, float* const f[8], cudaStream_t s) {
  const bool cfl = cfl_fused(F);
  if (F.wall) wall_launch(F, f, false, s);
  int rc = pre_div(F, f, s, cfl);
  if (rc) return rc;
  rc = launch_div(F, f, F.q, nullptr, 0.f, 0, 0, s, cfl);
  if (rc) return rc;
  courant_to_dev(F, f, s, cfl);
  STG_CUDA_OK(cudaGetLastError());
  return STAGGER_OK;
}

// A Courant-mode step is 38 to 50 launches whose arguments depend only on the
// state arrays and the context (the step dt lives on the device), so it is
// captured once, on a private stream, into a CUDA graph and replayed on the
// caller's stream: on small grids the launches, not the kernels, set the time.
// The capture is redone when the state arrays change, and not used while
// per-kernel timing is on; a failed capture falls back to direct launches.
int fused_step_graphed(Fused& F, float* f[8], double dt, cudaStream_t s) {
  if (dt > 0 || F.timing || F.step_state < 0) return fused_step(F, f, dt, s);
  bool same = F.step_state == 1;
  for (int c = 0; c < 8 && same; ++c) same = F.step_key[c] == f[c];
  if (!same) {
    if (!F.cap && cudaStreamCreateWithFlags(&F.cap, cudaStreamNonBlocking) != cudaSuccess) {
      F.cap = nullptr;
      F.step_state = -1;
      return fused_step(F, f, dt, s);
    }
    const long long l0 = F.launches;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool ok = cudaStreamBeginCapture(F.cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      const int rc = fused_step(F, f, dt, F.cap);
      ok = cudaStreamEndCapture(F.cap, &graph) == cudaSuccess && rc == STAGGER_OK && graph;
    }
    if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    const long long nl = F.launches - l0;
    F.launches = l0;
    if (!ok) {
      cudaGetLastError();   // clear a capture error; run the step directly from now on
      F.step_state = -1;
      return fused_step(F, f, dt, s);
    }
    if (F.step_exec) cudaGraphExecDestroy(F.step_exec);
    F.step_exec = exec;
    F.step_launches = nl;
    for (int c = 0; c < 8; ++c) F.step_key[c] = f[c];
    F.step_state = 1;
  }
  STG_CUDA_OK(cudaGraphLaunch(F.step_exec, s));
  F.launches += F.step_launches;
  return STAGGER_OK;
}

int fused_courant(Fused& F, float* const f[8], double lim[3], double* dt, cudaStream_t s) {
  int rc = fused_dt(F, f, s);
  if (rc) return rc;
  double h[4];
  STG_CUDA_OK(cudaMemcpyAsync(h, F.dt_dev, sizeof(h), cudaMemcpyDeviceToHost, s));
  STG_CUDA_OK(cudaStreamSynchronize(s));
  *dt = h[0];
  if (lim) { lim[0] = h[1]; lim[1] = h[2]; lim[2] = h[3]; }
  if (!(h[0] == h[0]) || h[0] <= 0) return STAGGER_ENONFINITE;
  return STAGGER_OK;
}

int fused_diagnostics(Fused& F, float* const f[8], const stagger_params& p, double out[10],
                      cudaStream_t s) {
  if (F.wall) wall_launch(F, f, false, s, false);
  dim3 gg = grid3(F.geo), bb(BX, BY, BZ);
  auto kdiag = F.zs ? k_diag_part<NbZ> : k_diag_part<Nb>;
  TIMED(K_DIAG, (kdiag<<<gg, bb, 0, s>>>(f[0], f[1], f[2], f[3], f[4], f[5], f[6], f[7], F.red,
                                         F.kp, F.geo)));
  STG_CUDA_OK(cudaGetLastError());
  std::vector<double> h((size_t)F.red_blocks * 10);
  STG_CUDA_OK(cudaMemcpyAsync(h.data(), F.red, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
  STG_CUDA_OK(cudaStreamSynchronize(s));
  double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = 0; b < F.red_blocks; ++b)
    for (int c = 0; c < 10; ++c)
      acc[c] = c == 7 ? fmax(acc[c], h[10 * b + c]) : acc[c] + h[10 * b + c];
  // Sums of the weights: every cell, or with closed z walls the physical
  // centre planes (half weight on the two boundary planes) and faces.
  // Rigid walls: every physical plane klo..khi once.
  const double N = F.wall == 1   ? (double)F.geo.sz * (F.kp.khi - F.kp.klo)
                   : F.wall >= 2 ? (double)F.geo.sz * (F.kp.khi - F.kp.klo + 1)
                                 : (double)F.geo.n;
  // Stellar-atmosphere boundaries: the z faces klo+1..khi.
  const double Nf = F.wall == 3 ? (double)F.geo.sz * (F.kp.khi - F.kp.klo) : N;
  out[0] = acc[0] + p.ref[0] * N;
  out[1] = acc[1] + p.ref[1] * N;
  out[2] = acc[2] + p.ref[2] * N;
  out[3] = acc[3] + p.ref[3] * (F.wall ? Nf : F.wsum_f);   // z-face weights on a stretched z
  out[4] = acc[4] + p.ref[4] * N;
  out[5] = acc[5];
  out[6] = acc[6];
  out[7] = acc[7];
  out[8] = sqrt(acc[8] / N);
  out[9] = acc[9];
  return acc[9] > 0 ? STAGGER_ENONFINITE : STAGGER_OK;
}

}  // namespace stg

// ===================================================== no-allocation entry ====
// stagger_diagnostics_noalloc: the diagnostics reduction with its scratch (the
// per-block FP64 partials and the ten final sums) in a fixed file-scope device
// array instead of memory from cudaMalloc.  The array is part of this
// library's device image, so every GPU that loads the library holds it until
// the process exits.  Limit: grids of at most NOALLOC_MAX_BLOCKS thread blocks
// of BX x BY x BZ = 32 x 2 x 4 cells (16,777,216 cells, e.g. 256^3).

namespace stg {

#define NOALLOC_MAX_BLOCKS 65536
#define NOALLOC_MAX_DEVICES 64
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_MAX_BLOCKS * 10 + 16];

// Device address of g_noalloc_scratch per device, as last looked up by
// cudaGetSymbolAddress (in host code the symbol names a host-side stand-in,
// not device memory).  It is looked up again on every call that is not being
// captured, so a context that was torn down and rebuilt (cudaDeviceReset)
// never sees a stale address; a captured call uses the stored one.
static double* g_noalloc_ptr[NOALLOC_MAX_DEVICES];

// Sum (max for entry 7) of the nb per-block partials into out[0..9], in a
// fixed order per thread and a fixed tree, so repeated calls agree bitwise.
__global__ void k_diag_final(const double* part, int nb, double* out) {
  __shared__ double sm[10][256];
  int tid = threadIdx.x;
  double v[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = tid; b < nb; b += blockDim.x)
    for (int c = 0; c < 10; ++c)
      v[c] = c == 7 ? fmax(v[c], part[10 * b + c]) : v[c] + part[10 * b + c];
  for (int c = 0; c < 10; ++c) sm[c][tid] = v[c];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (tid < s)
      for (int c = 0; c < 10; ++c)
        sm[c][tid] = c == 7 ? fmax(sm[c][tid], sm[c][tid + s]) : sm[c][tid] + sm[c][tid + s];
    __syncthreads();
  }
  if (tid < 10) out[tid] = sm[tid][0];
}

}  // namespace stg

extern "C" int stagger_diagnostics_noalloc(const stagger_grid* grid, const stagger_params* p,
                                           float* const state[8], double out[10],
                                           void* stream) {
  using namespace stg;
  if (!grid || !p || !state || !out) return STAGGER_EINVAL;
  for (int c = 0; c < 8; ++c)
    if (!state[c]) return STAGGER_EINVAL;
  // The same grid and parameter checks as stagger_create (sizes, launch-grid
  // limits, finiteness).  Every check, the stretched-z rejection included,
  // stays before the first launch: nothing below may run on arguments that a
  // check would have refused.
  int rc = validate_inputs(grid, p);
  if (rc) return rc;
  // A stretched z needs its mesh on the device, which this entry cannot
  // allocate; closed z walls need their ghost planes refilled (a launch on
  // the caller's state) and weighted sums: neither is offered here.
  if (p->zc || p->zf || p->zwalls) return STAGGER_EUNSUPPORTED;
  const long long nb = (((long long)grid->nx + BX - 1) / BX) * (((long long)grid->ny + BY - 1) / BY) *
                       (((long long)grid->nz + BZ - 1) / BZ);
  if (nb > NOALLOC_MAX_BLOCKS) return STAGGER_EINVAL;  // grid larger than the fixed scratch

  int dev = 0;
  STG_CUDA_OK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return STAGGER_EUNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  STG_CUDA_OK(cudaStreamIsCapturing(s, &cap));
  if (cap == cudaStreamCaptureStatusNone) {
    void* ptr = nullptr;
    STG_CUDA_OK(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_noalloc_ptr[dev] = (double*)ptr;
  } else if (!g_noalloc_ptr[dev]) {
    return STAGGER_EUNSUPPORTED;  // the first call on a device must not be captured
  }
  double* part = g_noalloc_ptr[dev];
  double* fin = part + (size_t)NOALLOC_MAX_BLOCKS * 10;

  // The kernel parameters the reduction reads (spacings, references, density
  // interpolation), from the caller's grid and parameters.
  KPar k;
  memset(&k, 0, sizeof(k));
  k.ih[0] = (float)(1.0 / grid->dx);
  k.ih[1] = (float)(1.0 / grid->dy);
  k.ih[2] = (float)(1.0 / grid->dz);
  k.r0 = (float)p->ref[0];
  k.r0pos = p->ref[0] > 0;
  for (int d = 0; d < 3; ++d) {
    k.pref[d] = (float)p->ref[1 + d];
    k.Bref[d] = (float)p->ref[5 + d];
  }
  k.log_interp = p->log_interp ? 1 : 0;
  Geo g = make_geo(grid->nx, grid->ny, grid->nz);
  dim3 gg = grid3(g), bb(BX, BY, BZ);
  // Each block writes all ten of its partials, so nothing carries over from
  // an earlier call.
  k_diag_part<Nb><<<gg, bb, 0, s>>>(state[0], state[1], state[2], state[3], state[4], state[5],
                                state[6], state[7], part, k, g);
  k_diag_final<<<1, 256, 0, s>>>(part, (int)nb, fin);
  STG_CUDA_OK(cudaGetLastError());
  double h[10];
  STG_CUDA_OK(cudaMemcpyAsync(h, fin, sizeof(h), cudaMemcpyDeviceToHost, s));
  STG_CUDA_OK(cudaStreamSynchronize(s));
  const double N = (double)g.n;
  for (int c = 0; c < 5; ++c) out[c] = h[c] + p->ref[c] * N;
  out[5] = h[5];
  out[6] = h[6];
  out[7] = h[7];
  out[8] = sqrt(h[8] / N);
  out[9] = h[9];
  return h[9] > 0 ? STAGGER_ENONFINITE : STAGGER_OK;
}
