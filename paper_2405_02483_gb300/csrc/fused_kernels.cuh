// Device code of the fused FP32 path (included by fused.cu).
#pragma once

#include <math.h>

#include "fused.cuh"

// Minimum resident blocks per SM requested from the register allocator
// (measured per kernel at 512^3: 4 for the wide flux/stress/divergence
// kernels, 8 where the tighter register budget was faster).
#ifndef STG_MINB
#define STG_MINB 4
#endif
#ifndef STG_MINB_HI
#define STG_MINB_HI 8
#endif

namespace stg {

// Thread block of the per-cell kernels: BX x BY x BZ cells.
#ifndef BX
#define BX 32
#endif
#ifndef BY
#define BY 2
#endif
#ifndef BZ
#define BZ 4
#endif

#define IA_ 0.5859375f
#define IB_ (-0.09765625f)
#define IC_ 0.01171875f
#define DA_ 1.171875f
#define DB_ (-0.065104166666666667f)
#define DC_ 0.0046875f

// Periodic neighbour offsets of one cell, offsets -3..3 per axis.
struct Nb {
  int c;
  int x[7];
  int y[7];
  int z[7];
  __device__ __forceinline__ int at(int dx, int dy, int dz) const {
    return z[dz + 3] + y[dy + 3] + x[dx + 3];
  }
  __device__ __forceinline__ int ax(int axis, int o) const {
    return axis == 0 ? at(o, 0, 0) : axis == 1 ? at(0, o, 0) : at(0, 0, o);
  }
};

__device__ __forceinline__ bool make_nb(Nb& n, const Geo& g) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= g.nx || j >= g.ny || k >= g.nz) return false;
#pragma unroll
  for (int o = -3; o <= 3; ++o) {
    n.x[o + 3] = wrap(i + o, g.nx);
    n.y[o + 3] = wrap(j + o, g.ny) * (int)g.sy;
    n.z[o + 3] = wrap(k + o, g.nz) * (int)g.sz;
  }
  n.c = n.z[3] + n.y[3] + n.x[3];
  return true;
}

// eq. (interp) to i+1/2 / i-1/2 and eq. (deriv) to i+1/2 / i-1/2, on a
// functor v(o) giving the operand at offset o along the stencil axis.
template <class V> __device__ __forceinline__ float s_up(V v) {
  return IA_ * (v(0) + v(1)) + IB_ * (v(-1) + v(2)) + IC_ * (v(-2) + v(3));
}
template <class V> __device__ __forceinline__ float s_dn(V v) {
  return IA_ * (v(-1) + v(0)) + IB_ * (v(-2) + v(1)) + IC_ * (v(-3) + v(2));
}
template <class V> __device__ __forceinline__ float s_du(V v, float ih) {
  return (DA_ * (v(1) - v(0)) + DB_ * (v(2) - v(-1)) + DC_ * (v(3) - v(-2))) * ih;
}
template <class V> __device__ __forceinline__ float s_dd(V v, float ih) {
  return (DA_ * (v(0) - v(-1)) + DB_ * (v(1) - v(-2)) + DC_ * (v(2) - v(-3))) * ih;
}

#define LDG(p, i) __ldg((p) + (i))
// Operand functors along one axis of a field at the thread's cell.
#define AX(fp, axis) [&](int o) { return LDG(fp, n.ax(axis, o)); }

__device__ __forceinline__ float dens(float t, const KPar& k) {
  if (k.log_interp) return k.r0pos ? k.r0 * expf(t) : expf(t);
  return k.r0 + t;
}

// ----------------------------------------------------------------- lr ------
__global__ void k_lr(const float* __restrict__ rd, float* __restrict__ lr, KPar k, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float r = rd[i];
  lr[i] = k.r0pos ? log1pf(r / k.r0) : logf(r);
}

// ------------------------------------------------------------- velocity ----
// u_d = p_d / rho_face with rho_face = dens(dn_d ls); the face values dn_d ls
// are also stored (lf, may be null) for the edge densities of the stresses.
__global__ void __launch_bounds__(BX * BY * BZ, STG_MINB) k_vel(
    const float* __restrict__ ls, const float* __restrict__ px, const float* __restrict__ py,
    const float* __restrict__ pz, float* __restrict__ ux, float* __restrict__ uy,
    float* __restrict__ uz, float* __restrict__ lfx, float* __restrict__ lfy,
    float* __restrict__ lfz, KPar k, Geo g) {
  Nb n;
  if (!make_nb(n, g)) return;
  const float lx = s_dn(AX(ls, 0)), ly = s_dn(AX(ls, 1)), lz = s_dn(AX(ls, 2));
  ux[n.c] = (LDG(px, n.c) + k.pref[0]) / dens(lx, k);
  uy[n.c] = (LDG(py, n.c) + k.pref[1]) / dens(ly, k);
  uz[n.c] = (LDG(pz, n.c) + k.pref[2]) / dens(lz, k);
  if (lfx) {
    lfx[n.c] = lx;
    lfy[n.c] = ly;
    lfz[n.c] = lz;
  }
}

// 2D interpolation up along a then b (edge -> centre) of f at the cell.
template <class N>
__device__ __forceinline__ float up2(const float* __restrict__ f, const N& n, int a, int b) {
  auto inner = [&](int oa) {
    auto v = [&](int ob) {
      int dx = (a == 0 ? oa : 0) + (b == 0 ? ob : 0);
      int dy = (a == 1 ? oa : 0) + (b == 1 ? ob : 0);
      int dz = (a == 2 ? oa : 0) + (b == 2 ? ob : 0);
      return LDG(f, n.at(dx, dy, dz));
    };
    return s_up(v);
  };
  return s_up(inner);
}

// ---------------------------------------------------------- viscosity ------
// Squared off-diagonal strain on the edges (Smagorinsky runs):
// S_xy^2 (Ez), S_yz^2 (Ex), S_zx^2 (Ey), S_ij = (dd_j u_i + dd_i u_j) / 2.
__global__ void __launch_bounds__(BX * BY * BZ, STG_MINB) k_strain2(
    const float* __restrict__ ux, const float* __restrict__ uy, const float* __restrict__ uz,
    float* __restrict__ sxy2, float* __restrict__ syz2, float* __restrict__ szx2, KPar k, Geo g) {
  Nb n;
  if (!make_nb(n, g)) return;
  const float* ih = k.ih;
  float sxy = 0.5f * (s_dd(AX(ux, 1), ih[1]) + s_dd(AX(uy, 0), ih[0]));
  float syz = 0.5f * (s_dd(AX(uy, 2), ih[2]) + s_dd(AX(uz, 1), ih[1]));
  float szx = 0.5f * (s_dd(AX(uz, 0), ih[0]) + s_dd(AX(ux, 2), ih[2]));
  sxy2[n.c] = sxy * sxy;
  syz2[n.c] = syz * syz;
  szx2[n.c] = szx * szx;
}

// eq. (RMnu): nu1 |u| + nu3 (c_s + c_A) + nu2 dl_min max(0, -div u), centred.
template <bool SMAG>
__global__ void __launch_bounds__(BX * BY * BZ, SMAG ? STG_MINB : STG_MINB_HI) k_nu_raw(
    const float* __restrict__ ux,
                                                const float* __restrict__ uy,
                                                const float* __restrict__ uz,
                                                const float* __restrict__ rd,
                                                const float* __restrict__ Ed,
                                                const float* __restrict__ bx,
                                                const float* __restrict__ by,
                                                const float* __restrict__ bz,
                                                const float* __restrict__ sqxy,
                                                const float* __restrict__ sqyz,
                                                const float* __restrict__ sqzx,
                                                float* __restrict__ nv, KPar k, Geo g) {
  Nb n;
  if (!make_nb(n, g)) return;
  float ucx = s_up(AX(ux, 0)), ucy = s_up(AX(uy, 1)), ucz = s_up(AX(uz, 2));
  const float sxx = s_du(AX(ux, 0), k.ih[0]), syy = s_du(AX(uy, 1), k.ih[1]),
              szz = s_du(AX(uz, 2), k.ih[2]);
  float divu = sxx + syy + szz;
  float nu = 0.f;
  if (k.nu1 > 0.f) nu = k.nu1 * sqrtf(ucx * ucx + ucy * ucy + ucz * ucz);
  if (k.nu3 > 0.f) {
    float bcx = s_up(AX(bx, 0)) + k.Bref[0], bcy = s_up(AX(by, 1)) + k.Bref[1],
          bcz = s_up(AX(bz, 2)) + k.Bref[2];
    float r = LDG(rd, n.c) + k.r0;
    float P = k.gm1 * (LDG(Ed, n.c) + k.E0);
    float cs = sqrtf(k.gamma * P / r);
    float ca = sqrtf((bcx * bcx + bcy * bcy + bcz * bcz) / r);
    nu += k.nu3 * (cs + ca);
  }
  if (k.nu2dl > 0.f) nu += k.nu2dl * fmaxf(-divu, 0.f);
  if (SMAG) {
    // eq. (nusmag): dl_min Csmag [2 (S_ii^2 - (div u)^2/3 + S_ij^2, i != j)]^1/2.
    float s2 = ((sxx * sxx + syy * syy) + szz * szz) - divu * divu * (1.f / 3.f);
    s2 += 2.f * ((up2(sqxy, n, 0, 1) + up2(sqyz, n, 1, 2)) + up2(sqzx, n, 2, 0));
    nu += k.csmag_dl * sqrtf(2.f * fmaxf(s2, 0.f));
  }
  nv[n.c] = nu;
}

// 3-cell max along x, y and z: the maximum over the 3x3x3 neighbourhood.
__global__ void __launch_bounds__(BX * BY * BZ, STG_MINB) k_nu_max(const float* __restrict__ a,
                                                float* __restrict__ b, Geo g) {
  Nb n;
  if (!make_nb(n, g)) return;
  float m = -INFINITY;
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) m = fmaxf(m, LDG(a, n.at(dx, dy, dz)));
  b[n.c] = m;
}

// 3-cell mean along x, y and z (the 3x3x3 mean) and its logarithm.
__global__ void __launch_bounds__(BX * BY * BZ, STG_MINB_HI) k_nu_smooth(const float* __restrict__ a,
                                                   float* __restrict__ nu,
                                                   float* __restrict__ lnu, Geo g) {
  Nb n;
  if (!make_nb(n, g)) return;
  float sz = 0.f;
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz) {
    float sy = 0.f;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      float sx = LDG(a, n.at(-1, dy, dz)) + LDG(a, n.at(0, dy, dz)) + LDG(a, n.at(1, dy, dz));
      sy += sx;
    }
    sz += sy;
  }
  float v = sz * (1.f / 27.f);
  nu[n.c] = v;
  lnu[n.c] = logf(fmaxf(v, 1e-30f));
}

// ln<nu> interpolated to the three faces (first half of the edge values).
__global__ void __launch_bounds__(BX * BY * BZ, STG_MINB) k_nu_faces(
    const float* __restrict__ lnu, float* __restrict__ lx, float* __restrict__ ly,
    float* __restrict__ lz, Geo g) {
  Nb n;
  if (!make_nb(n, g)) return;
  lx[n.c] = s_dn(AX(lnu, 0));
  ly[n.c] = s_dn(AX(lnu, 1));
  lz[n.c] = s_dn(AX(lnu, 2));
}

// -------------------------------------------------------------- stress -----
// Strain, stress (eq. (itv)), J = curl B and eta J on edges, eq. (ohm).
__global__ void __launch_bounds__(BX * BY * BZ, STG_MINB) k_tau(
    const float* __restrict__ ux, const float* __restrict__ uy, const float* __restrict__ uz,
    const float* __restrict__ rd, const float* __restrict__ lfx, const float* __restrict__ lfy,
    const float* __restrict__ lfz, const float* __restrict__ nu, const float* __restrict__ lnx,
    const float* __restrict__ lny, const float* __restrict__ lnz,
    const float* __restrict__ bx, const float* __restrict__ by,
    const float* __restrict__ bz, float* __restrict__ txx, float* __restrict__ tyy,
    float* __restrict__ tzz, float* __restrict__ txy, float* __restrict__ tyz,
    float* __restrict__ tzx, float* __restrict__ Rx, float* __restrict__ Ry,
    float* __restrict__ Rz, float* __restrict__ Jx, float* __restrict__ Jy,
    float* __restrict__ Jz, KPar k, Geo g) {
  Nb n;
  if (!make_nb(n, g)) return;
  const float* ih = k.ih;
  float jx = s_dd(AX(bz, 1), ih[1]) - s_dd(AX(by, 2), ih[2]);
  float jy = s_dd(AX(bx, 2), ih[2]) - s_dd(AX(bz, 0), ih[0]);
  float jz = s_dd(AX(by, 0), ih[0]) - s_dd(AX(bx, 1), ih[1]);
  Jx[n.c] = jx;
  Jy[n.c] = jy;
  Jz[n.c] = jz;
  if (!k.visc) return;
  float sxx = s_du(AX(ux, 0), ih[0]), syy = s_du(AX(uy, 1), ih[1]), szz = s_du(AX(uz, 2), ih[2]);
  float divu = (sxx + syy) + szz;
  float r = LDG(rd, n.c) + k.r0;
  float nuc = k.rm ? LDG(nu, n.c) : 0.f;
  float nxx = k.rm ? k.sp[0] * nuc : k.nu_const;
  float nyy = k.rm ? k.sp[1] * nuc : k.nu_const;
  float nzz = k.rm ? k.sp[2] * nuc : k.nu_const;
  txx[n.c] = (r * nxx) * (sxx + k.c1 * divu);
  tyy[n.c] = (r * nyy) * (syy + k.c1 * divu);
  tzz[n.c] = (r * nzz) * (szz + k.c1 * divu);
  // Edge values: the second interpolation of the face values (Ex edge from
  // the y faces along z, Ey from the z faces along x, Ez from the x faces along y).
  float nyz = k.rm ? k.spp[0] * expf(s_dn(AX(lny, 2))) : k.nu_const;
  float nzx = k.rm ? k.spp[1] * expf(s_dn(AX(lnz, 0))) : k.nu_const;
  float nxy = k.rm ? k.spp[2] * expf(s_dn(AX(lnx, 1))) : k.nu_const;
  float ryz = dens(s_dn(AX(lfy, 2)), k), rzx = dens(s_dn(AX(lfz, 0)), k),
        rxy = dens(s_dn(AX(lfx, 1)), k);
  float sxy = 0.5f * (s_dd(AX(ux, 1), ih[1]) + s_dd(AX(uy, 0), ih[0]));
  float syz = 0.5f * (s_dd(AX(uy, 2), ih[2]) + s_dd(AX(uz, 1), ih[1]));
  float szx = 0.5f * (s_dd(AX(uz, 0), ih[0]) + s_dd(AX(ux, 2), ih[2]));
  txy[n.c] = (rxy * nxy) * sxy;
  tyz[n.c] = (ryz * nyz) * syz;
  tzx[n.c] = (rzx * nzx) * szx;
  Rx[n.c] = (k.nuB * nyz) * jx;
  Ry[n.c] = (k.nuB * nzx) * jy;
  Rz[n.c] = (k.nuB * nxy) * jz;
}

// eq. (quench): T <- T min(max over the axes a0, a1 of max3(q), qlim),
// q = |d2 T| / (M + |d2 T| / qmax), M the 3-cell max of |T| along the axis.
template <class N>
__device__ __forceinline__ float quench1(const float* __restrict__ T, const N& n, int a0, int a1,
                                         const KPar& k) {
  float fac = -1.f;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    int a = t == 0 ? a0 : a1;
    if (a < 0) continue;
    float v[5];
#pragma unroll
    for (int o = -2; o <= 2; ++o) v[o + 2] = LDG(T, n.ax(a, o));
    float m = -1.f;
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      float d2 = (v[o + 2] - 2.f * v[o + 1]) + v[o];
      float a2 = fabsf(d2);
      float M = fmaxf(fmaxf(fabsf(v[o]), fabsf(v[o + 1])), fabsf(v[o + 2]));
      float q = a2 / ((M + a2 * k.inv_qmax) + 1e-30f);
      m = fmaxf(m, q);
    }
    fac = fmaxf(fac, m);
  }
  return LDG(T, n.c) * fminf(fac, k.qlim);
}

// Quenched stresses, the quenched resistive field eta J (left in the E arrays,
// where k_flux adds -u x B) and the heating densities
// w_c = sum tau_ii S_ii (centre), w_edge = 2 tau_ij S_ij + eta J . J (edge).
// Viscous runs only.
__global__ void __launch_bounds__(BX * BY * BZ, STG_MINB_HI) k_edge(
    const float* __restrict__ txx, const float* __restrict__ tyy, const float* __restrict__ tzz,
    const float* __restrict__ txy, const float* __restrict__ tyz, const float* __restrict__ tzx,
    const float* __restrict__ Rx, const float* __restrict__ Ry, const float* __restrict__ Rz,
    const float* __restrict__ Jx, const float* __restrict__ Jy, const float* __restrict__ Jz,
    const float* __restrict__ ux, const float* __restrict__ uy, const float* __restrict__ uz,
    float* __restrict__ qxx, float* __restrict__ qyy, float* __restrict__ qzz,
    float* __restrict__ qxy, float* __restrict__ qyz, float* __restrict__ qzx,
    float* __restrict__ Ex, float* __restrict__ Ey, float* __restrict__ Ez,
    float* __restrict__ wc, float* __restrict__ wx, float* __restrict__ wy,
    float* __restrict__ wz, KPar k, Geo g) {
  Nb n;
  if (!make_nb(n, g)) return;
  float txx_, tyy_, tzz_, txy_, tyz_, tzx_, rx_, ry_, rz_;
  if (k.do_quench) {
    txx_ = quench1(txx, n, 0, -1, k);
    tyy_ = quench1(tyy, n, 1, -1, k);
    tzz_ = quench1(tzz, n, 2, -1, k);
    txy_ = quench1(txy, n, 0, 1, k);
    tyz_ = quench1(tyz, n, 1, 2, k);
    tzx_ = quench1(tzx, n, 2, 0, k);
    rx_ = quench1(Rx, n, 1, 2, k);
    ry_ = quench1(Ry, n, 2, 0, k);
    rz_ = quench1(Rz, n, 0, 1, k);
    qxx[n.c] = txx_;
    qyy[n.c] = tyy_;
    qzz[n.c] = tzz_;
    qxy[n.c] = txy_;
    qyz[n.c] = tyz_;
    qzx[n.c] = tzx_;
  } else {
    txx_ = LDG(txx, n.c); tyy_ = LDG(tyy, n.c); tzz_ = LDG(tzz, n.c);
    txy_ = LDG(txy, n.c); tyz_ = LDG(tyz, n.c); tzx_ = LDG(tzx, n.c);
    rx_ = LDG(Rx, n.c); ry_ = LDG(Ry, n.c); rz_ = LDG(Rz, n.c);
  }
  Ex[n.c] = rx_;
  Ey[n.c] = ry_;
  Ez[n.c] = rz_;
  const float* ih = k.ih;
  float sxx = s_du(AX(ux, 0), ih[0]), syy = s_du(AX(uy, 1), ih[1]), szz = s_du(AX(uz, 2), ih[2]);
  float sxy = 0.5f * (s_dd(AX(ux, 1), ih[1]) + s_dd(AX(uy, 0), ih[0]));
  float syz = 0.5f * (s_dd(AX(uy, 2), ih[2]) + s_dd(AX(uz, 1), ih[1]));
  float szx = 0.5f * (s_dd(AX(uz, 0), ih[0]) + s_dd(AX(ux, 2), ih[2]));
  wc[n.c] = (txx_ * sxx + tyy_ * syy) + tzz_ * szz;
  wx[n.c] = 2.f * (tyz_ * syz) + rx_ * LDG(Jx, n.c);
  wy[n.c] = 2.f * (tzx_ * szx) + ry_ * LDG(Jy, n.c);
  wz[n.c] = 2.f * (txy_ * sxy) + rz_ * LDG(Jz, n.c);
}

// ---------------------------------------------------------------- flux -----
struct FluxIn {
  const float *px, *py, *pz, *rd, *Ed, *bx, *by, *bz, *ls, *ux, *uy, *uz;
  const float *qxx, *qyy, *qzz, *qxy, *qyz, *qzx, *Jx, *Jy, *Jz, *nu, *wc, *wx, *wy, *wz;
};
struct FluxOut {
  float *mxx, *myy, *mzz, *mxy, *myx, *mxz, *mzx, *myz, *mzy;
  float *lx1, *lx2, *ly1, *ly2, *lz1, *lz2, *gx, *gy, *gz, *qt;
  float *ex, *ey, *ez;   // in: eta J (viscous runs); out: E = -u x B + eta J
};


template <class N>
__device__ __forceinline__ void flux_cell(const N& n, const FluxIn& in, const FluxOut& out,
                                          const KPar& k) {
  const float* pr[3] = {in.px, in.py, in.pz};
  const float* uu[3] = {in.ux, in.uy, in.uz};
  const float* qd[3] = {in.qxx, in.qyy, in.qzz};
  float* md[3] = {out.mxx, out.myy, out.mzz};
  const float Pd = k.gm1 * LDG(in.Ed, n.c);
  // Diagonal momentum flux at centres: up(p_d) up(u_d) + P - tau_dd.
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float* pp = pr[d];
    const float* up_ = uu[d];
    float v = (s_up(AX(pp, d)) + k.pref[d]) * s_up(AX(up_, d)) + Pd;
    if (k.visc) v -= LDG(qd[d], n.c);
    md[d][n.c] = v;
  }
  // The twelve edge interpolations of u and B, shared by the off-diagonal
  // momentum fluxes, the Lorentz products and -u x B.
  const float* B0 = k.Bref;
  const float uy_z = s_dn(AX(in.uy, 2)), uz_y = s_dn(AX(in.uz, 1));   // Ex edge
  const float bz_y = s_dn(AX(in.bz, 1)) + B0[2], by_z = s_dn(AX(in.by, 2)) + B0[1];
  const float uz_x = s_dn(AX(in.uz, 0)), ux_z = s_dn(AX(in.ux, 2));   // Ey edge
  const float bx_z = s_dn(AX(in.bx, 2)) + B0[0], bz_x = s_dn(AX(in.bz, 0)) + B0[2];
  const float ux_y = s_dn(AX(in.ux, 1)), uy_x = s_dn(AX(in.uy, 0));   // Ez edge
  const float by_x = s_dn(AX(in.by, 0)) + B0[1], bx_y = s_dn(AX(in.bx, 1)) + B0[0];
  // Off-diagonal: p_d carried along axis a, at the (d, a) edge.
  auto off = [&](int d, int a, float ua, const float* tau) {
    const float* pp = pr[d];
    float v = (s_dn(AX(pp, a)) + k.pref[d]) * ua;
    if (k.visc) v -= LDG(tau, n.c);
    return v;
  };
  out.mxy[n.c] = off(0, 1, uy_x, in.qxy);
  out.myx[n.c] = off(1, 0, ux_y, in.qxy);
  out.mxz[n.c] = off(0, 2, uz_x, in.qzx);
  out.mzx[n.c] = off(2, 0, ux_z, in.qzx);
  out.myz[n.c] = off(1, 2, uz_y, in.qyz);
  out.mzy[n.c] = off(2, 1, uy_z, in.qyz);
  // Lorentz force pieces J_a dn_d(B_b) on edges.
  const float jx = LDG(in.Jx, n.c), jy = LDG(in.Jy, n.c), jz = LDG(in.Jz, n.c);
  out.lx1[n.c] = jy * bz_x;
  out.lx2[n.c] = jz * by_x;
  out.ly1[n.c] = jz * bx_y;
  out.ly2[n.c] = jx * bz_y;
  out.lz1[n.c] = jx * by_z;
  out.lz2[n.c] = jy * bx_z;
  // E = -u x B (eq. ohm) plus the quenched eta J left by k_edge.
  const float ex = -((uy_z * bz_y) - (uz_y * by_z));
  const float ey = -((uz_x * bx_z) - (ux_z * bz_x));
  const float ez = -((ux_y * by_x) - (uy_x * bx_y));
  out.ex[n.c] = k.visc ? ex + out.ex[n.c] : ex;
  out.ey[n.c] = k.visc ? ey + out.ey[n.c] : ey;
  out.ez[n.c] = k.visc ? ez + out.ez[n.c] : ez;
  // Energy fluxes p_d dn(e) - nuE dn(rho nu_dd) dddn(e) at faces.
  float* go[3] = {out.gx, out.gy, out.gz};
  const float* rd = in.rd;
  const float* Ed = in.Ed;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    auto e_at = [&](int o) {
      int i = n.ax(d, o);
      return (LDG(Ed, i) + k.E0) / (LDG(rd, i) + k.r0);
    };
    float v = (LDG(pr[d], n.c) + k.pref[d]) * s_dn(e_at);
    if (k.visc) {
      auto ed_at = [&](int o) {
        int i = n.ax(d, o);
        float r = LDG(rd, i) + k.r0;
        return (LDG(Ed, i) - k.e0 * LDG(rd, i)) / r;
      };
      auto rn_at = [&](int o) {
        int i = n.ax(d, o);
        float r = LDG(rd, i) + k.r0;
        return r * (k.rm ? k.sp[d] * LDG(in.nu, i) : k.nu_const);
      };
      v -= k.nuE * (s_dn(rn_at) * s_dd(ed_at, k.ih[d]));
    }
    go[d][n.c] = v;
  }
  // -P div u + Q, Q = w_c + up up of the edge heating densities.
  float divu = (s_du(AX(in.ux, 0), k.ih[0]) + s_du(AX(in.uy, 1), k.ih[1])) +
               s_du(AX(in.uz, 2), k.ih[2]);
  float P = k.gm1 * (LDG(Ed, n.c) + k.E0);
  float qt = -P * divu;
  if (k.visc) {
    float Q = LDG(in.wc, n.c) + ((up2(in.wz, n, 0, 1) + up2(in.wx, n, 1, 2)) + up2(in.wy, n, 2, 0));
    qt += Q;
  }
  if (k.inv_tcool > 0.f) {
    // Newtonian cooling, eq. (NewtonCool), per volume: -rho (e - e_cool) / t_cool,
    // times the density cutoff of eq. (rhocool).
    const float r = LDG(in.rd, n.c) + k.r0;
    float qn = -((LDG(Ed, n.c) + k.E0) - r * k.e_cool) * k.inv_tcool;
    if (k.cool_cut) {
      const float x = r * k.inv_rho_cool, x2 = x * x;
      qn *= (k.cool_cut == 1 ? x2 : 1.f) / (1.f + x2);
    }
    qt += qn;
  }
  out.qt[n.c] = qt;
}

__global__ void __launch_bounds__(BX * BY * BZ, STG_MINB) k_flux(FluxIn in, FluxOut out, KPar k, Geo g) {
  Nb n;
  if (!make_nb(n, g)) return;
  flux_cell(n, in, out, k);
}

// ----------------------------------------------------------- divergence ----
struct DivIn {
  const float *px, *py, *pz;
  const float *mxx, *myy, *mzz, *mxy, *myx, *mxz, *mzx, *myz, *mzy;
  const float *lx1, *lx2, *ly1, *ly2, *lz1, *lz2, *gx, *gy, *gz, *qt, *Ex, *Ey, *Ez, *ls;
  const float* f[8];   // stage input (deviations), for the update
};

// F(f) and the RK update: q <- alpha q + F, f_out <- f + beta dt q.
// mode 0: write F to q only; 1: also update with dt from *dtp.
__global__ void __launch_bounds__(BX * BY * BZ, STG_MINB) k_div(DivIn in, float* q0, float* q1, float* q2, float* q3,
                                             float* q4, float* q5, float* q6, float* q7,
                                             float* o0, float* o1, float* o2, float* o3,
                                             float* o4, float* o5, float* o6, float* o7,
                                             float alpha, float beta, const double* dtp,
                                             int mode, KPar k, Geo g) {
  Nb n;
  if (!make_nb(n, g)) return;
  const float* ih = k.ih;
  float F[8];
  F[0] = -((s_du(AX(in.px, 0), ih[0]) + s_du(AX(in.py, 1), ih[1])) + s_du(AX(in.pz, 2), ih[2]));
  float t;
  t = -s_dd(AX(in.mxx, 0), ih[0]);
  t -= s_du(AX(in.mxy, 1), ih[1]);
  t -= s_du(AX(in.mxz, 2), ih[2]);
  t += s_up(AX(in.lx1, 2));
  t -= s_up(AX(in.lx2, 1));
  if (k.g[0] != 0.f) t += dens(s_dn(AX(in.ls, 0)), k) * k.g[0];
  F[1] = t;
  t = -s_du(AX(in.myx, 0), ih[0]);
  t -= s_dd(AX(in.myy, 1), ih[1]);
  t -= s_du(AX(in.myz, 2), ih[2]);
  t += s_up(AX(in.ly1, 0));
  t -= s_up(AX(in.ly2, 2));
  if (k.g[1] != 0.f) t += dens(s_dn(AX(in.ls, 1)), k) * k.g[1];
  F[2] = t;
  t = -s_du(AX(in.mzx, 0), ih[0]);
  t -= s_du(AX(in.mzy, 1), ih[1]);
  t -= s_dd(AX(in.mzz, 2), ih[2]);
  t += s_up(AX(in.lz1, 1));
  t -= s_up(AX(in.lz2, 0));
  if (k.g[2] != 0.f) t += dens(s_dn(AX(in.ls, 2)), k) * k.g[2];
  F[3] = t;
  F[4] = -((s_du(AX(in.gx, 0), ih[0]) + s_du(AX(in.gy, 1), ih[1])) + s_du(AX(in.gz, 2), ih[2])) +
         LDG(in.qt, n.c);
  F[5] = -(s_du(AX(in.Ez, 1), ih[1]) - s_du(AX(in.Ey, 2), ih[2]));
  F[6] = -(s_du(AX(in.Ex, 2), ih[2]) - s_du(AX(in.Ez, 0), ih[0]));
  F[7] = -(s_du(AX(in.Ey, 0), ih[0]) - s_du(AX(in.Ex, 1), ih[1]));
  float* qs[8] = {q0, q1, q2, q3, q4, q5, q6, q7};
  float* os[8] = {o0, o1, o2, o3, o4, o5, o6, o7};
  float bdt = mode ? (float)((double)beta * dtp[0]) : 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    float qq = alpha != 0.f ? alpha * qs[c][n.c] + F[c] : F[c];
    qs[c][n.c] = qq;
    if (mode) os[c][n.c] = LDG(in.f[c], n.c) + bdt * qq;
  }
}

__global__ void k_set_dt(double* dtp, double dt) { dtp[0] = dt; }

// f_out = f + beta dt q for the 8 fields in one launch (blockIdx.y = field),
// 16-byte vectors when every array is 16-byte aligned and n % 4 == 0.
struct Upd8 {
  const float* f[8];
  const float* q[8];
  float* o[8];
};
__global__ void k_update8(Upd8 u, float beta, const double* dtp, long long n, int vec) {
  const int c = blockIdx.y;
  const float bdt = (float)((double)beta * dtp[0]);
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (vec) {
    const float4* f = reinterpret_cast<const float4*>(u.f[c]);
    const float4* q = reinterpret_cast<const float4*>(u.q[c]);
    float4* o = reinterpret_cast<float4*>(u.o[c]);
    for (; i < n / 4; i += stride) {
      float4 a = __ldg(f + i), b = __ldg(q + i);
      o[i] = make_float4(a.x + bdt * b.x, a.y + bdt * b.y, a.z + bdt * b.z, a.w + bdt * b.w);
    }
  } else {
    for (; i < n; i += stride) u.o[c][i] = __ldg(u.f[c] + i) + bdt * __ldg(u.q[c] + i);
  }
}

// f_out = f + beta dt q (stage-1 update once the Courant step is known).
__global__ void k_update(const float* __restrict__ f, const float* __restrict__ q,
                         float* __restrict__ o, float beta, const double* dtp, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  o[i] = f[i] + (float)((double)beta * dtp[0]) * q[i];
}

// -------------------------------------------------------------- Courant ----
// Per-cell wave speed c_s + c_A + |u_perp|, rate max(|dr/dt|/r, |dE/dt|/E)
// and <nu>; block maxima to part[3*block + {0,1,2}] (as doubles).
__global__ void __launch_bounds__(BX * BY * BZ, STG_MINB_HI) k_courant_part(
    const float* __restrict__ ux, const float* __restrict__ uy, const float* __restrict__ uz,
    const float* __restrict__ rd, const float* __restrict__ Ed, const float* __restrict__ bx,
    const float* __restrict__ by, const float* __restrict__ bz, const float* __restrict__ qr,
    const float* __restrict__ qE, const float* __restrict__ nu, double* part, KPar k, Geo g) {
  __shared__ float sm[3][BX * BY * BZ];
  Nb n;
  float w = 0.f, rate = 0.f, nuv = 0.f;
  int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
  if (make_nb(n, g)) {
    float ucx = s_up(AX(ux, 0)), ucy = s_up(AX(uy, 1)), ucz = s_up(AX(uz, 2));
    float bcx = s_up(AX(bx, 0)) + k.Bref[0], bcy = s_up(AX(by, 1)) + k.Bref[1],
          bcz = s_up(AX(bz, 2)) + k.Bref[2];
    float r = LDG(rd, n.c) + k.r0;
    float E = LDG(Ed, n.c) + k.E0;
    float cs = sqrtf(k.gamma * (k.gm1 * E) / r);
    float B2 = bcx * bcx + bcy * bcy + bcz * bcz;
    float ca = sqrtf(B2 / r);
    float u2 = ucx * ucx + ucy * ucy + ucz * ucz;
    float ub = ucx * bcx + ucy * bcy + ucz * bcz;
    float up2 = B2 > 0.f ? u2 - ub * ub / B2 : u2;
    w = cs + ca + sqrtf(fmaxf(up2, 0.f));
    rate = fmaxf(fabsf(LDG(qr, n.c)) / r, fabsf(LDG(qE, n.c)) / E);
    if (k.visc) nuv = k.rm ? LDG(nu, n.c) : k.nu_const;
    // A NaN anywhere must survive the max: map it to +inf.
    if (!(w == w)) w = INFINITY;
    if (!(rate == rate)) rate = INFINITY;
    if (!(nuv == nuv)) nuv = INFINITY;
  }
  sm[0][tid] = w;
  sm[1][tid] = rate;
  sm[2][tid] = nuv;
  __syncthreads();
  for (int s = BX * BY * BZ / 2; s > 0; s >>= 1) {
    if (tid < s)
      for (int c = 0; c < 3; ++c) sm[c][tid] = fmaxf(sm[c][tid], sm[c][tid + s]);
    __syncthreads();
  }
  if (tid == 0) {
    int b = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    for (int c = 0; c < 3; ++c) part[3 * b + c] = (double)sm[c][0];
  }
}

// Final FP64 reduction: dt = min(Cdt dl/wmax, Cdtr/ratemax, Cdtd dl/(numax f)).
__global__ void k_courant_final(const double* part, int nb, double* dt_out, double cdt,
                                double cdtr, double cdtd, double dlmin, double dfac,
                                int nu_is_velocity) {
  __shared__ double sm[3][256];
  int tid = threadIdx.x;
  double m[3] = {0, 0, 0};
  for (int b = tid; b < nb; b += blockDim.x)
    for (int c = 0; c < 3; ++c) m[c] = fmax(m[c], part[3 * b + c]);
  for (int c = 0; c < 3; ++c) sm[c][tid] = m[c];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (tid < s)
      for (int c = 0; c < 3; ++c) sm[c][tid] = fmax(sm[c][tid], sm[c][tid + s]);
    __syncthreads();
  }
  if (tid == 0) {
    double wmax = sm[0][0], rmax = sm[1][0], nmax = sm[2][0];
    double tw = wmax > 0 ? cdt * dlmin / wmax : HUGE_VAL;
    double tr = rmax > 0 ? cdtr / rmax : HUGE_VAL;
    double nv = nu_is_velocity ? nmax : nmax / dlmin;
    double td = nv > 0 ? cdtd * dlmin / (nv * dfac) : HUGE_VAL;
    double dt = fmin(tw, fmin(tr, td));
    dt_out[0] = dt;
    dt_out[1] = tw;
    dt_out[2] = tr;
    dt_out[3] = td;
  }
}

// ---------------------------------------------------------- diagnostics ----
// Per-block FP64 partials: sum r', px', py', pz', E', kinetic, magnetic,
// max |div B|, sum (div B)^2, non-finite count.
__global__ void __launch_bounds__(BX * BY * BZ, STG_MINB) k_diag_part(
    const float* __restrict__ rd, const float* __restrict__ px, const float* __restrict__ py,
    const float* __restrict__ pz, const float* __restrict__ Ed, const float* __restrict__ bx,
    const float* __restrict__ by, const float* __restrict__ bz, double* part, KPar k, Geo g) {
  __shared__ double sm[10][BX * BY * BZ];
  Nb n;
  double v[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
  if (make_nb(n, g)) {
    const float* pr[3] = {px, py, pz};
    const float* bb[3] = {bx, by, bz};
    float vals[8] = {LDG(rd, n.c), LDG(px, n.c), LDG(py, n.c), LDG(pz, n.c),
                     LDG(Ed, n.c), LDG(bx, n.c), LDG(by, n.c), LDG(bz, n.c)};
    int bad = 0;
    for (int c = 0; c < 8; ++c) bad += isfinite(vals[c]) ? 0 : 1;
    v[0] = vals[0];
    v[1] = vals[1];
    v[2] = vals[2];
    v[3] = vals[3];
    v[4] = vals[4];
    double kin = 0, mag = 0, divb = 0;
    for (int d = 0; d < 3; ++d) {
      auto lsv = [&](int o) {
        float r = LDG(rd, n.ax(d, o));
        if (!k.log_interp) return r;
        return k.r0pos ? log1pf(r / k.r0) : logf(r);
      };
      double rf = (double)dens(s_dn(lsv), k);
      double p = (double)LDG(pr[d], n.c) + k.pref[d];
      kin += 0.5 * p * p / rf;
      double b = (double)LDG(bb[d], n.c) + k.Bref[d];
      mag += 0.5 * b * b;
      const float* bp = bb[d];
      divb += (double)s_du(AX(bp, d), k.ih[d]);
    }
    v[5] = kin;
    v[6] = mag;
    v[7] = fabs(divb);
    v[8] = divb * divb;
    v[9] = bad;
  }
  for (int c = 0; c < 10; ++c) sm[c][tid] = v[c];
  __syncthreads();
  for (int s = BX * BY * BZ / 2; s > 0; s >>= 1) {
    if (tid < s)
      for (int c = 0; c < 10; ++c)
        sm[c][tid] = c == 7 ? fmax(sm[c][tid], sm[c][tid + s]) : sm[c][tid] + sm[c][tid + s];
    __syncthreads();
  }
  if (tid == 0) {
    int b = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    for (int c = 0; c < 10; ++c) part[10 * b + c] = sm[c][0];
  }
}


}  // namespace stg
