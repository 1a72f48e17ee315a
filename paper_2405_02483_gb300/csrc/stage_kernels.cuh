// Fused flux-divergence stage kernel (included by fused.cu after
// fused_kernels.cuh), the layout stagger_params.fuse_flux_div = 1 selects.
//
// k_fdiv takes the place of the materialised-flux part of an RK stage (k_flux,
// k_flux_e, k_cool2 and the three k_div launches): every momentum, Lorentz,
// induction and energy flux of eqs. (mom), (ien), (ohm) is formed on chip and
// consumed by the divergences of eqs. (mass), (mom), (ien), (indu) and the
// low-storage update of eqs. (ddt), (tupdate) in the same kernel, so no flux
// array reaches HBM.
//
// Layout.  A block of FD_TX x TY threads owns an FD_TX x TY column tile of
// the (x, y) plane, one cell per thread, and marches along z through a chunk
// of FD_ZC planes.  At each flux plane m:
//   * every owner thread forms all fluxes at its own cell of plane m (the
//     centre, the three edges, the three faces) by gathers from the stage's
//     input arrays;
//   * the fluxes that are differentiated in the plane (along x or y) go to a
//     shared-memory plane with a 3-cell halo; the halo strips are formed by
//     the block's threads as extra tasks (the 3 x TY strips left and right
//     for the x-differentiated fluxes, the FD_TX x 3 strips above and below
//     for the y-differentiated ones);
//   * the fluxes that are differentiated or interpolated along z are not
//     stored: each is multiplied by its stencil weights and added at once to
//     the pending right-hand sides of the seven output planes m-3 .. m+3 it
//     reaches, held in registers (semi-stencil accumulation).  Output plane
//     m-3 is then complete, is combined with the previous derivative and the
//     stage input (the RK update), and is written.
// Each input array is read from HBM about once per plane and only the
// derivative and the updated state are written.  The price is one cell per
// thread (the z accumulators of four cells would not fit the registers) and
// the recomputed halo strips: on GB300 at 512^3 the kernel executes about 1.5
// times the instructions per cell of the split kernels, whose four-cell
// threads load 16 bytes at a time, and is slower than they are, so the split
// layout is the default.

namespace stg {

#ifndef FD_ZC
#define FD_ZC 64
#endif
#define FD_TX 32
#define FD_W (FD_TX + 6)   // tile width with its x halo

// Inputs of one stage: the stage state and the per-cell primitives formed
// by k_lr_ed and k_vel, plus, in viscous runs, the (quenched) stresses, the
// (quenched) resistive field eta J, <nu> and the heating densities of k_edge.
struct FdIn {
  const float* f[8];              // stage input state (deviations), r px py pz E Bx By Bz
  const float *ux, *uy, *uz;      // face velocities
  const float* ed;                // e - e0 at centres
  const float* ler;               // ln e - ln <e>_h (ediffav)
  const float* ls;                // ln(rho/r0) (log interpolation) or rho' (gravity)
  const float *txx, *tyy, *tzz, *txy, *tyz, *tzx;   // stresses (viscous)
  const float *rx, *ry, *rz;      // eta J on the edges (viscous)
  const float *nu, *wc, *wx, *wy, *wz;               // <nu>, heating densities (viscous)
};

// Which fluxes a task forms: all (the owner of a cell), the y-differentiated
// ones with Ez (a task of the y halo), the x-differentiated ones with Ez
// (a task of the x halo), or only those differentiated or interpolated along
// z (the owner on the planes before and after its chunk).
enum { FD_OWN = 0, FD_YS = 1, FD_XS = 2, FD_Z = 3 };

// Shared-memory planes: x-differentiated fluxes, y-differentiated fluxes, Ez.
enum { SX_MXX = 0, SX_MYX, SX_LY1, SX_MZX, SX_LZ2, SX_GX, SX_EY,
       SY_MXY, SY_LX2, SY_MYY, SY_MZY, SY_LZ1, SY_GY, SY_EX, S_EZ, S_COUNT };

struct FdFlux {
  float mxx, myy, mzz, qt;          // centre
  float mxy, myx, lx2, ly1, ez;     // Ez edge (i-1/2, j-1/2, k)
  float myz, mzy, ly2, lz1, ex;     // Ex edge (i, j-1/2, k-1/2)
  float mxz, mzx, lx1, lz2, ey;     // Ey edge (i-1/2, j, k-1/2)
  float gx, gy, gz;                 // faces
};

// Operand functors over a shared-memory flux plane along x and along y.
struct SmX {
  const float* p;
  __device__ __forceinline__ float operator()(int o) const { return p[o]; }
};
struct SmY {
  const float* p;
  __device__ __forceinline__ float operator()(int o) const { return p[o * FD_W]; }
};

// Neighbour offsets of cell (i, j, k), all periodic.
__device__ __forceinline__ void fd_nb_xy(Nb& n, const Geo& g, int i, int j) {
#pragma unroll
  for (int o = -3; o <= 3; ++o) {
    n.x[o + 3] = wrap(i + o, g.nx);
    n.y[o + 3] = wrap(j + o, g.ny) * (int)g.sy;
  }
}
__device__ __forceinline__ void fd_nb_z(Nb& n, const Geo& g, int k) {
#pragma unroll
  for (int o = -3; o <= 3; ++o) n.z[o + 3] = wrap(k + o, g.nz) * (int)g.sz;
  n.c = n.z[3] + n.y[3] + n.x[3];
  n.kz = wrap(k, g.nz);
}

// The fluxes of eqs. (mom), (ien), (ohm) at one cell, as k_flux and k_flux_e
// form them (reading R1 for the centrings), with J = curl B formed here from
// the field.  WHO selects the subset.
template <int WHO, bool VISC>
__device__ __forceinline__ void fd_fluxes(const Nb& n, const FdIn& in, const KPar& k, FdFlux& o) {
  const float* px = in.f[1];
  const float* py = in.f[2];
  const float* pz = in.f[3];
  const float* bx = in.f[5];
  const float* by = in.f[6];
  const float* bz = in.f[7];
  const float* B0 = k.Bref;
  // X: x-differentiated, Y: y-differentiated, Z: z-differentiated fluxes.
  constexpr bool X = WHO == FD_OWN || WHO == FD_XS, Y = WHO == FD_OWN || WHO == FD_YS,
                 Z = WHO == FD_OWN || WHO == FD_Z;
  const float Pd = k.gm1 * n.ld(in.f[4]);
  // Centre: up(p_d) up(u_d) + P - tau_dd.
  if (X) {
    o.mxx = (s_up(AX(px, 0)) + k.pref[0]) * s_up(AX(in.ux, 0)) + Pd;
    if (VISC) o.mxx -= n.ld(in.txx);
  }
  if (Y) {
    o.myy = (s_up(AX(py, 1)) + k.pref[1]) * s_up(AX(in.uy, 1)) + Pd;
    if (VISC) o.myy -= n.ld(in.tyy);
  }
  if (Z) {
    o.mzz = (s_up(AX(pz, 2)) + k.pref[2]) * s_up(AX(in.uz, 2)) + Pd;
    if (VISC) o.mzz -= n.ld(in.tzz);
  }
  if (X || Y) {  // Ez edge
    const float ux_y = s_dn(AX(in.ux, 1)), uy_x = s_dn(AX(in.uy, 0));
    const float by_x = s_dn(AX(by, 0)) + B0[1], bx_y = s_dn(AX(bx, 1)) + B0[0];
    const float jz = s_dd(AX(by, 0), k.ih[0]) - s_dd(AX(bx, 1), k.ih[1]);
    const float t = VISC ? n.ld(in.txy) : 0.f;
    if (Y) {
      o.mxy = (s_dn(AX(px, 1)) + k.pref[0]) * uy_x - t;
      o.lx2 = jz * by_x;
    }
    if (X) {
      o.myx = (s_dn(AX(py, 0)) + k.pref[1]) * ux_y - t;
      o.ly1 = jz * bx_y;
    }
    o.ez = -((ux_y * by_x) - (uy_x * bx_y));
    if (VISC) o.ez += n.ld(in.rz);
  }
  if (Y || Z) {  // Ex edge
    const float uy_z = s_dn(AX(in.uy, 2)), uz_y = s_dn(AX(in.uz, 1));
    const float bz_y = s_dn(AX(bz, 1)) + B0[2], by_z = s_dn(AX(by, 2)) + B0[1];
    const float jx = s_dd(AX(bz, 1), k.ih[1]) - s_dd(AX(by, 2), k.ih[2]);
    const float t = VISC ? n.ld(in.tyz) : 0.f;
    if (Z) {
      o.myz = (s_dn(AX(py, 2)) + k.pref[1]) * uz_y - t;
      o.ly2 = jx * bz_y;
    }
    if (Y) {
      o.mzy = (s_dn(AX(pz, 1)) + k.pref[2]) * uy_z - t;
      o.lz1 = jx * by_z;
    }
    o.ex = -((uy_z * bz_y) - (uz_y * by_z));
    if (VISC) o.ex += n.ld(in.rx);
  }
  if (X || Z) {  // Ey edge
    const float uz_x = s_dn(AX(in.uz, 0)), ux_z = s_dn(AX(in.ux, 2));
    const float bx_z = s_dn(AX(bx, 2)) + B0[0], bz_x = s_dn(AX(bz, 0)) + B0[2];
    const float jy = s_dd(AX(bx, 2), k.ih[2]) - s_dd(AX(bz, 0), k.ih[0]);
    const float t = VISC ? n.ld(in.tzx) : 0.f;
    if (Z) {
      o.mxz = (s_dn(AX(px, 2)) + k.pref[0]) * uz_x - t;
      o.lx1 = jy * bz_x;
    }
    if (X) {
      o.mzx = (s_dn(AX(pz, 0)) + k.pref[2]) * ux_z - t;
      o.lz2 = jy * bx_z;
    }
    o.ey = -((uz_x * bx_z) - (ux_z * bz_x));
    if (VISC) o.ey += n.ld(in.ry);
  }
  // Energy fluxes p_d dn(e) - nuE dn(rho nu_dd) dddn(e) at the faces; e = e0 +
  // (e - e0), the interpolation weights summing to one.
  auto gflux = [&](int d, const float* pd) {
    auto ed_at = [&](int oo) { return n.lda(in.ed, d, oo); };
    const float ef = s_dn(ed_at) + k.e0;
    float v = (n.ld(pd) + k.pref[d]) * ef;
    if (VISC) {
      auto rn_at = [&](int oo) {
        const float r = n.lda(in.f[0], d, oo) + k.r0;
        return r * (k.rm ? k.sp[d] * n.lda(in.nu, d, oo) : k.nu_const);
      };
      if (k.ediffav) {   // eq. (ediffav)
        auto le_at = [&](int oo) { return n.lda(in.ler, d, oo); };
        v -= k.nuE * (s_dn(rn_at) * (ef * s_dd(le_at, k.ih[d])));
      } else {
        v -= k.nuE * (s_dn(rn_at) * s_dd(ed_at, k.ih[d]));
      }
    }
    return v;
  };
  if (X) o.gx = gflux(0, px);
  if (Y) o.gy = gflux(1, py);
  if (Z) o.gz = gflux(2, pz);
}

// The pointwise part of the energy equation at the owner's centre: -P div u,
// the centre heating density and the in-plane (x then y) part of its edge
// terms, and the cooling terms of eqs. (NewtonCool), (ChromoCool), (CoronaCool).
template <bool VISC>
__device__ __forceinline__ float fd_qt(const Nb& n, const FdIn& in, const KPar& k) {
  const float divu = (s_du(AX(in.ux, 0), k.ih[0]) + s_du(AX(in.uy, 1), k.ih[1])) +
                     s_du(AX(in.uz, 2), k.ih[2]);
  const float Ev = n.ld(in.f[4]);
  float qt = -(k.gm1 * (Ev + k.E0)) * divu;
  if (VISC) qt += n.ld(in.wc) + up2(in.wz, n, 0, 1);
  if (k.inv_tcool > 0.f || k.inv_tchromo > 0.f || k.corL0 > 0.f) {
    const float rdv = n.ld(in.f[0]);
    const float r = rdv + k.r0;
    if (k.inv_tcool > 0.f) {
      float qn = -((Ev + k.E0) - r * k.e_cool) * k.inv_tcool;
      if (k.cool_cut) {
        const float x = r * k.inv_rho_cool, x2 = x * x;
        qn *= (k.cool_cut == 1 ? x2 : 1.f) / (1.f + x2);
      }
      qt += qn;
    }
    if (k.inv_tchromo > 0.f) {
      const float edv = fdiv((Ev + k.Ec) - k.e0 * rdv, r);
      const float x = r * k.inv_rhobot;
      const float x53 = x * cbrtf(x) * cbrtf(x);
      qt -= (r * x53) * ((edv - (float)k.emean[n.kz]) * k.inv_tchromo);
    }
    if (k.corL0 > 0.f) {
      const float Tk = (k.corTu * k.gm1) * fdiv(Ev + k.E0, r);
      const float t4 = Tk * 1e-4f;
      qt -= (k.corL0 * (r * r)) * (expf(-(t4 * t4)) * rsqrtf(Tk));
    }
  }
  return qt;
}

// Weights of the z stencils applied to a value at plane m and added to the
// output plane m - 3 + s (slot s of the accumulators): d/dz up (eq. (deriv),
// face -> centre) at slots 0..5, d/dz dn (centre -> face) at slots 1..6, the
// interpolation up (eq. (interp)) at slots 0..5.
#define FD_WDU(s) ((s) == 0 ? DC_ : (s) == 1 ? DB_ : (s) == 2 ? DA_ : (s) == 3 ? -DA_ : (s) == 4 ? -DB_ : -DC_)
#define FD_WDD(s) ((s) == 1 ? DC_ : (s) == 2 ? DB_ : (s) == 3 ? DA_ : (s) == 4 ? -DA_ : (s) == 5 ? -DB_ : -DC_)
#define FD_WUP(s) ((s) == 0 ? IC_ : (s) == 1 ? IB_ : (s) == 2 ? IA_ : (s) == 3 ? IA_ : (s) == 4 ? IB_ : IC_)

#ifndef FD_MINB
#define FD_MINB 2
#endif
// Dynamic shared memory of k_fdiv for a tile of TY rows.
constexpr size_t fd_smem_bytes(int ty) { return sizeof(float) * S_COUNT * (ty + 6) * FD_W; }

template <int TY, bool VISC, bool CR>
__global__ void __launch_bounds__(FD_TX * TY, TY <= 8 ? FD_MINB : 1) k_fdiv(
    FdIn in, float* q0, float* q1, float* q2, float* q3, float* q4, float* q5, float* q6,
    float* q7, float* o0, float* o1, float* o2, float* o3, float* o4, float* o5, float* o6,
    float* o7, float alpha, const float* bdtp, int mode, unsigned* cr, KPar k,
    Geo g) {
  static_assert(6 * FD_TX + 6 * TY <= FD_TX * TY, "one halo task per thread");
  // S_COUNT flux planes of (TY + 6) x FD_W floats (dynamic shared memory).
  extern __shared__ float fd_smem[];
  auto sm = reinterpret_cast<float(*)[TY + 6][FD_W]>(fd_smem);
  float* const qs[8] = {q0, q1, q2, q3, q4, q5, q6, q7};
  float* const os[8] = {o0, o1, o2, o3, o4, o5, o6, o7};
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * FD_TX + tx;
  const int x0 = blockIdx.x * FD_TX, y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * FD_ZC;
  const int z1 = min(z0 + FD_ZC, g.nz);
  const int i = x0 + tx, j = y0 + ty;
  const bool own = i < g.nx && j < g.ny;   // an output cell (else only smem fluxes)
  const float bdt = mode ? bdtp[0] : 0.f;
  const float ihz = k.ih[2];
  // With a single plane every z-derivative and z-interpolation difference is
  // exactly zero (periodic wrap of size 1): the z parts are left out rather
  // than summed to a rounding residue.
  const bool zact = g.nz > 1;

  // Halo task of this thread: first the y strips (FD_TX x 3 above and below),
  // then the x strips (3 x TY left and right).
  const int ny_tasks = 6 * FD_TX, nx_tasks = 6 * TY;
  int hr = -1, hc = -1, hkind = 0;
  if (tid < ny_tasks) {
    const int rr = tid / FD_TX;
    hr = rr < 3 ? rr : TY + rr;
    hc = 3 + tid % FD_TX;
    hkind = FD_YS;
  } else if (tid < ny_tasks + nx_tasks) {
    const int u = tid - ny_tasks;
    const int cc = u % 6;
    hc = cc < 3 ? cc : FD_TX + cc;
    hr = 3 + u / 6;
    hkind = FD_XS;
  }
  Nb nh, n;
  if (hkind) fd_nb_xy(nh, g, wrap(x0 - 3 + hc, g.nx), wrap(y0 - 3 + hr, g.ny));
  fd_nb_xy(n, g, wrap(i, g.nx), wrap(j, g.ny));

  // Pending right-hand sides of the output planes m-3 .. m+3 (slot s: plane
  // m - 3 + s).  Equations with d/dz up or up_z terms reach slots 0..5, the
  // z momentum (d/dz dn) slots 0..6, Bz (in-plane terms only) slots 0..3.
  float ar[6], apx[6], apy[6], apz[7], aE[6], aBx[6], aBy[6], aBz[4];
#pragma unroll
  for (int s = 0; s < 6; ++s) ar[s] = apx[s] = apy[s] = aE[s] = aBx[s] = aBy[s] = 0.f;
#pragma unroll
  for (int s = 0; s < 7; ++s) apz[s] = 0.f;
#pragma unroll
  for (int s = 0; s < 4; ++s) aBz[s] = 0.f;
  unsigned mb = 0u;

  for (int m = z0 - 3; m <= z1 + 2; ++m) {
    const bool inplane = m >= z0 && m < z1;
    fd_nb_z(n, g, m);
    FdFlux fo;
    if (inplane) {
      fd_fluxes<FD_OWN, VISC>(n, in, k, fo);
      const int r0 = ty + 3, c0 = tx + 3;
      sm[SX_MXX][r0][c0] = fo.mxx; sm[SX_MYX][r0][c0] = fo.myx; sm[SX_LY1][r0][c0] = fo.ly1;
      sm[SX_MZX][r0][c0] = fo.mzx; sm[SX_LZ2][r0][c0] = fo.lz2; sm[SX_GX][r0][c0] = fo.gx;
      sm[SX_EY][r0][c0] = fo.ey;
      sm[SY_MXY][r0][c0] = fo.mxy; sm[SY_LX2][r0][c0] = fo.lx2; sm[SY_MYY][r0][c0] = fo.myy;
      sm[SY_MZY][r0][c0] = fo.mzy; sm[SY_LZ1][r0][c0] = fo.lz1; sm[SY_GY][r0][c0] = fo.gy;
      sm[SY_EX][r0][c0] = fo.ex; sm[S_EZ][r0][c0] = fo.ez;
      if (hkind) {
        fd_nb_z(nh, g, m);
        FdFlux fh;
        if (hkind == FD_YS) {
          fd_fluxes<FD_YS, VISC>(nh, in, k, fh);
          sm[SY_MXY][hr][hc] = fh.mxy; sm[SY_LX2][hr][hc] = fh.lx2; sm[SY_MYY][hr][hc] = fh.myy;
          sm[SY_MZY][hr][hc] = fh.mzy; sm[SY_LZ1][hr][hc] = fh.lz1; sm[SY_GY][hr][hc] = fh.gy;
          sm[SY_EX][hr][hc] = fh.ex; sm[S_EZ][hr][hc] = fh.ez;
        } else {
          fd_fluxes<FD_XS, VISC>(nh, in, k, fh);
          sm[SX_MXX][hr][hc] = fh.mxx; sm[SX_MYX][hr][hc] = fh.myx; sm[SX_LY1][hr][hc] = fh.ly1;
          sm[SX_MZX][hr][hc] = fh.mzx; sm[SX_LZ2][hr][hc] = fh.lz2; sm[SX_GX][hr][hc] = fh.gx;
          sm[SX_EY][hr][hc] = fh.ey; sm[S_EZ][hr][hc] = fh.ez;
        }
      }
    } else if (own && zact) {
      // Warm-up and tail planes: only the fluxes differentiated along z.
      fd_fluxes<FD_Z, VISC>(n, in, k, fo);
    }
    // up_z(up_y(wx)) and up_z(up_x(wy)) of eqs. (vdiss), (ien): their in-plane
    // interpolation here, the z one through the accumulators.
    float wq = 0.f;
    if (VISC && own && (zact || inplane)) wq = s_up(AX(in.wx, 1)) + s_up(AX(in.wy, 0));
    if (own && !zact && inplane) {
      // A single plane: the z-derivatives vanish and each z-interpolation is
      // the weighted sum of six copies of the value.
      auto up1 = [](float v) { return s_up([v](int) { return v; }); };
      apx[3] += up1(fo.lx1);
      apy[3] -= up1(fo.ly2);
      if (VISC) aE[3] += up1(wq);
    }
    if (own && zact) {
      // z parts: d/dz up of pz, mxz, myz, gz, Ey, Ex; d/dz dn of mzz; up_z of
      // lx1, ly2 (and of the in-plane halves of the edge heating densities).
      const float fpz = n.ld(in.f[3]);
#pragma unroll
      for (int s = 0; s < 6; ++s) {
        const float wu = FD_WDU(s) * ihz, wi = FD_WUP(s);
        ar[s] -= wu * fpz;
        apx[s] += wi * fo.lx1 - wu * fo.mxz;
        apy[s] -= wi * fo.ly2 + wu * fo.myz;
        aE[s] -= wu * fo.gz;
        if (VISC) aE[s] += wi * wq;
        aBx[s] += wu * fo.ey;
        aBy[s] -= wu * fo.ex;
      }
#pragma unroll
      for (int s = 1; s < 7; ++s) apz[s] -= FD_WDD(s) * ihz * fo.mzz;
    }
    __syncthreads();
    if (inplane && own) {
      const int r0 = ty + 3, c0 = tx + 3;
      auto X = [&](int f) { return SmX{&sm[f][r0][c0]}; };
      auto Y = [&](int f) { return SmY{&sm[f][r0][c0]}; };
      const float ihx = k.ih[0], ihy = k.ih[1];
      ar[3] -= s_du(AX(in.f[1], 0), ihx) + s_du(AX(in.f[2], 1), ihy);
      float t = -s_dd(X(SX_MXX), ihx) - s_du(Y(SY_MXY), ihy) - s_up(Y(SY_LX2));
      float u = -s_du(X(SX_MYX), ihx) - s_dd(Y(SY_MYY), ihy) + s_up(X(SX_LY1));
      float v = -s_du(X(SX_MZX), ihx) - s_du(Y(SY_MZY), ihy) + s_up(Y(SY_LZ1)) - s_up(X(SX_LZ2));
      if (k.g[0] != 0.f) t += dens(s_dn(AX(in.ls, 0)), k) * k.g[0];
      if (k.g[1] != 0.f) u += dens(s_dn(AX(in.ls, 1)), k) * k.g[1];
      if (k.g[2] != 0.f) v += dens(s_dn(AX(in.ls, 2)), k) * k.g[2];
      apx[3] += t;
      apy[3] += u;
      apz[3] += v;
      aE[3] += fd_qt<VISC>(n, in, k) - (s_du(X(SX_GX), ihx) + s_du(Y(SY_GY), ihy));
      aBx[3] -= s_du(Y(S_EZ), ihy);
      aBy[3] += s_du(X(S_EZ), ihx);
      aBz[3] += s_du(Y(SY_EX), ihy) - s_du(X(SX_EY), ihx);
    }
    __syncthreads();
    // Output plane m - 3 is complete: RK update, eqs. (ddt), (tupdate).
    const int ko = m - 3;
    if (own && ko >= z0) {
      const long long c = (long long)ko * g.sz + (long long)j * g.sy + i;
      // Rigid z walls (R25): the time derivatives of the ghost planes are zero.
      const bool fz = k.wall == 2 && (ko < k.klo || ko > k.khi);
      const float F[8] = {fz ? 0.f : ar[0], fz ? 0.f : apx[0], fz ? 0.f : apy[0],
                          fz ? 0.f : apz[0], fz ? 0.f : aE[0], fz ? 0.f : aBx[0],
                          fz ? 0.f : aBy[0], fz ? 0.f : aBz[0]};
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float qq = alpha != 0.f ? alpha * qs[e][c] + F[e] : F[e];
        qs[e][c] = qq;
        if (mode) os[e][c] = __ldg(in.f[e] + c) + bdt * qq;
      }
      if (CR) {
        const float r = __ldg(in.f[0] + c) + k.r0, E = __ldg(in.f[4] + c) + k.E0;
        mb = max(mb, max_bits(fmaxf(fabsf(F[0]) / r, fabsf(F[4]) / E)));
      }
    }
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      ar[s] = ar[s + 1]; apx[s] = apx[s + 1]; apy[s] = apy[s + 1];
      aE[s] = aE[s + 1]; aBx[s] = aBx[s + 1]; aBy[s] = aBy[s + 1];
    }
    ar[5] = apx[5] = apy[5] = aE[5] = aBx[5] = aBy[5] = 0.f;
#pragma unroll
    for (int s = 0; s < 6; ++s) apz[s] = apz[s + 1];
    apz[6] = 0.f;
#pragma unroll
    for (int s = 0; s < 3; ++s) aBz[s] = aBz[s + 1];
    aBz[3] = 0.f;
  }
  if constexpr (CR) block_max_to<FD_TX * TY>(mb, cr);
}

}  // namespace stg
