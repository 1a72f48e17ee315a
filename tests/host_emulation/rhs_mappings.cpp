// Host build of the fused kernels: the right-hand side formed by the stage
// kernels with one cell per thread (Nb) equals the one formed with four
// x-cells per thread (Nb4, with the z-marching k_nu_maxsmooth in place of
// k_nu_max + k_nu_smooth, as on the device) bit for bit, for two parameter
// sets: RM viscosity with the quench, and every option at once (Smagorinsky
// with RM, the bulk term, gravity, no log interpolation, the second-order
// switch, Newtonian, chromospheric and coronal cooling).  Exit status: the
// number of (case, shape) pairs that differ.
#include <cuda_runtime.h>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>
#undef __global__
#undef __device__
#undef __host__
#undef __forceinline__
#undef __launch_bounds__
#undef __shared__
#define __global__
#define __device__
#define __host__
#define __forceinline__ inline
#define __launch_bounds__(...)
#define __shared__ static
#define __ldg(p) (*(p))
#define __syncthreads()
uint3 blockIdx, threadIdx;
dim3 blockDim, gridDim;
static inline float __fdividef(float a, float b) { return a / b; }
static inline float rsqrtf(float x) { return 1.f / sqrtf(x); }
static inline float __uint_as_float(unsigned u) { float f; memcpy(&f, &u, 4); return f; }
static inline unsigned __float_as_uint(float f) { unsigned u; memcpy(&u, &f, 4); return u; }
static inline unsigned max(unsigned a, unsigned b) { return a > b ? a : b; }
static inline int min(int a, int b) { return a < b ? a : b; }
static inline unsigned __shfl_xor_sync(unsigned, unsigned v, int) { return v; }
static inline unsigned atomicMax(unsigned* p, unsigned v) {
  unsigned o = *p;
  if (v > o) *p = v;
  return o;
}
#include "../../paper_2405_02483_gb300/csrc/fused_kernels.cuh"
using namespace stg;

template <class K>
static void run(dim3 gd, dim3 bd, K kern) {
  gridDim = gd;
  blockDim = bd;
  for (unsigned bz = 0; bz < gd.z; ++bz)
    for (unsigned by = 0; by < gd.y; ++by)
      for (unsigned bx = 0; bx < gd.x; ++bx)
        for (unsigned tz = 0; tz < bd.z; ++tz)
          for (unsigned ty = 0; ty < bd.y; ++ty)
            for (unsigned tx = 0; tx < bd.x; ++tx) {
              blockIdx = make_uint3(bx, by, bz);
              threadIdx = make_uint3(tx, ty, tz);
              kern();
            }
}
template <class N, class K>
static void launch(const Geo& g, K kern) {
  run(dim3((g.nx + BX * N::W - 1) / (BX * N::W), (g.ny + BY - 1) / BY, (g.nz + BZ - 1) / BZ),
      dim3(BX, BY, BZ), kern);
}

struct Case {
  float nu1, nu2, nu3, nuE, nuB, c1, csmag, g2, tcool, ecool, rhocool, tchromo, rhobot, corL0, corTu;
  int quench, log_interp, cool_cut, d2div;
  float d2lim;
};

// The stage's kernels in the device's order; f: eight FP32 deviations.
template <class N>
static void rhs(const Geo& g, const KPar& kin, float* const* f, std::vector<std::vector<float>>& d,
                std::vector<unsigned char>& flag, float* const* out) {
  KPar k = kin;
  for (auto& a : d) std::fill(a.begin(), a.end(), 0.f);
  std::vector<double> em(g.nz, 0.0);
  for (int kz = 0; kz < g.nz; ++kz) {
    double acc = 0;
    for (long long i = 0; i < (long long)g.nx * g.ny; ++i) {
      const long long c = kz * (long long)g.nx * g.ny + i;
      acc += (double)(((f[4][c] + k.Ec) - k.e0 * f[0][c]) / (f[0][c] + k.r0));
    }
    em[kz] = acc / ((double)g.nx * g.ny);
  }
  k.emean = em.data();
  float* D[F_COUNT];
  for (int i = 0; i < F_COUNT; ++i) D[i] = d[i].data();
  const float* ls = k.log_interp ? D[F_LR] : f[0];
  using NB = typename N::Base;
  run(dim3((unsigned)((g.n / N::W + 255) / 256)), dim3(256), [&] {
    k_lr_ed<NB>(f[0], f[4], k.log_interp ? D[F_LR] : nullptr, D[F_ED], nullptr, nullptr, k, g.n,
                g.sz);
  });
  launch<N>(g, [&] { k_vel<NB>(ls, f[1], f[2], f[3], D[F_UX], D[F_UY], D[F_UZ], D[F_LFX], D[F_LFY], D[F_LFZ], k, g); });
  if (k.rm) {
    if (k.csmag_dl > 0.f) {
      launch<N>(g, [&] { k_strain2<N>(D[F_UX], D[F_UY], D[F_UZ], D[F_SQXY], D[F_SQYZ], D[F_SQZX], k, g); });
      launch<N>(g, [&] {
        k_nu_raw<true, false, N>(D[F_UX], D[F_UY], D[F_UZ], f[0], f[4], f[5], f[6], f[7], D[F_SQXY],
                                 D[F_SQYZ], D[F_SQZX], D[F_NV], nullptr, k, g);
      });
    } else {
      launch<N>(g, [&] {
        k_nu_raw<false, false, N>(D[F_UX], D[F_UY], D[F_UZ], f[0], f[4], f[5], f[6], f[7], D[F_SQXY],
                                  D[F_SQYZ], D[F_SQZX], D[F_NV], nullptr, k, g);
      });
    }
    if (N::W == 4) {
      run(dim3((g.nx + 127) / 128, (g.ny + NUZ_TY - 1) / NUZ_TY, (g.nz + NUZ_ZC - 1) / NUZ_ZC), dim3(32, NUZ_TY),
          [&] { k_nu_maxsmooth<false>(D[F_NV], D[F_NU], D[F_LNU], nullptr, g); });
    } else {
      launch<N>(g, [&] { k_nu_max<NB>(D[F_NV], D[F_NM], g); });
      launch<N>(g, [&] { k_nu_smooth<NB, false>(D[F_NM], D[F_NU], D[F_LNU], nullptr, g); });
    }
    launch<N>(g, [&] { k_nu_faces<NB>(D[F_LNU], D[F_LNX], D[F_LNY], D[F_LNZ], g); });
  }
  unsigned char* fl = flag.data();
  if (k.d2div) launch<N>(g, [&] { k_d2flag<NB>(f[0], f[4], fl, k, g); });
  auto ktau = k.d2div ? k_tau<N, true> : k_tau<N, false>;
  launch<N>(g, [&] {
    ktau(D[F_UX], D[F_UY], D[F_UZ], f[0], D[F_LFX], D[F_LFY], D[F_LFZ], D[F_NU], D[F_LNX], D[F_LNY],
         D[F_LNZ], f[5], f[6], f[7], D[F_TXX], D[F_TYY], D[F_TZZ], D[F_TXY], D[F_TYZ], D[F_TZX], D[F_RX],
         D[F_RY], D[F_RZ], D[F_JX], D[F_JY], D[F_JZ], fl, k, g);
  });
  auto kedge = k.d2div ? k_edge<N, true> : k_edge<N, false>;
  if (k.visc)
    launch<N>(g, [&] {
      kedge(D[F_TXX], D[F_TYY], D[F_TZZ], D[F_TXY], D[F_TYZ], D[F_TZX], D[F_RX], D[F_RY], D[F_RZ], D[F_JX],
            D[F_JY], D[F_JZ], D[F_UX], D[F_UY], D[F_UZ], D[F_QXX], D[F_QYY], D[F_QZZ], D[F_QXY], D[F_QYZ],
            D[F_QZX], D[F_EX], D[F_EY], D[F_EZ], D[F_WC], D[F_WX], D[F_WY], D[F_WZ], fl, k, g);
    });
  const bool qn = k.visc && k.do_quench;
  FluxIn fi = {f[1], f[2], f[3], f[0], f[4], f[5], f[6], f[7], ls, D[F_UX], D[F_UY], D[F_UZ],
               qn ? D[F_QXX] : D[F_TXX], qn ? D[F_QYY] : D[F_TYY], qn ? D[F_QZZ] : D[F_TZZ],
               qn ? D[F_QXY] : D[F_TXY], qn ? D[F_QYZ] : D[F_TYZ], qn ? D[F_QZX] : D[F_TZX],
               D[F_JX], D[F_JY], D[F_JZ], D[F_NU], D[F_WC], D[F_WX], D[F_WY], D[F_WZ], D[F_ED]};
  FluxOut fo = {D[F_MXX], D[F_MYY], D[F_MZZ], D[F_MXY], D[F_MYX], D[F_MXZ], D[F_MZX], D[F_MYZ],
                D[F_MZY], D[F_LX1], D[F_LX2], D[F_LY1], D[F_LY2], D[F_LZ1], D[F_LZ2], D[F_GX],
                D[F_GY], D[F_GZ], D[F_QT], D[F_EX], D[F_EY], D[F_EZ]};
  launch<N>(g, [&] { k_flux<N>(fi, fo, k, g); });
  launch<N>(g, [&] { k_flux_e<N>(fi, fo, k, g); });
  if (k.inv_tchromo > 0.f || k.corL0 > 0.f) launch<N>(g, [&] { k_cool2<NB>(f[0], f[4], D[F_QT], k, g); });
  DivIn di;
  di.px = f[1]; di.py = f[2]; di.pz = f[3];
  di.mxx = D[F_MXX]; di.myy = D[F_MYY]; di.mzz = D[F_MZZ]; di.mxy = D[F_MXY]; di.myx = D[F_MYX];
  di.mxz = D[F_MXZ]; di.mzx = D[F_MZX]; di.myz = D[F_MYZ]; di.mzy = D[F_MZY];
  di.lx1 = D[F_LX1]; di.lx2 = D[F_LX2]; di.ly1 = D[F_LY1]; di.ly2 = D[F_LY2];
  di.lz1 = D[F_LZ1]; di.lz2 = D[F_LZ2];
  di.gx = D[F_GX]; di.gy = D[F_GY]; di.gz = D[F_GZ]; di.qt = D[F_QT];
  di.Ex = D[F_EX]; di.Ey = D[F_EY]; di.Ez = D[F_EZ]; di.ls = ls;
  di.lq = D[F_LQ];
  di.uz = D[F_UZ];
  for (int c = 0; c < 8; ++c) di.f[c] = f[c];
  float bdtv = 0;
  launch<N>(g, [&] {
    k_div<N, 0xFF, false>(di, out[0], out[1], out[2], out[3], out[4], out[5], out[6], out[7], out[0], out[1],
                          out[2], out[3], out[4], out[5], out[6], out[7], 0.f, &bdtv, 0, nullptr, k, g);
  });
}

int main() {
  const Case cases[2] = {
      // RM viscosity with the quench (the benchmark's physics)
      {0.04f, 1.f, 0.04f, 1.f, 1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 1.f, 0.f, 1.f, 0.f, 1.f, 1, 1, 0, 0, 0.3f},
      // every option at once
      {0.04f, 1.f, 0.04f, 1.f, 0.8f, -1.f / 3.f, 0.15f, -0.5f, 0.2f, 0.8f, 1.1f, 0.08f, 0.9f, 1.f, 8e3f, 1, 0, 1, 1,
       0.3f},
  };
  const int shapes[][3] = {{16, 8, 6}, {20, 4, 5}, {8, 3, 7}, {132, 2, 3}};
  int bad = 0;
  for (int stretched = 0; stretched < 2; ++stretched)
  for (int ci = 0; ci < 2; ++ci) {
    const Case& C = cases[ci];
    for (const auto& sh : shapes) {
      const int nx = sh[0], ny = sh[1], nz = sh[2];
      const Geo g = make_geo(nx, ny, nz);
      std::mt19937 rng(nx * 131 + ny * 17 + nz + ci);
      std::uniform_real_distribution<float> U(-1.f, 1.f);
      const float amp[8] = {0.1f, 0.5f, 0.5f, 0.5f, 0.1f, 0.3f, 0.3f, 0.3f};
      std::vector<std::vector<float>> st(8, std::vector<float>(g.n));
      for (int c = 0; c < 8; ++c)
        for (auto& v : st[c]) v = amp[c] * U(rng);
      float* f[8];
      for (int c = 0; c < 8; ++c) f[c] = st[c].data();
      KPar k;
      memset(&k, 0, sizeof(k));
      const double h[3] = {1.0 / nx, 1.1 / ny, 0.9 / nz};
      const double dlmin = std::min(h[0], std::min(h[1], h[2]));
      for (int a = 0; a < 3; ++a) { k.ih[a] = (float)(1.0 / h[a]); k.sp[a] = (float)h[a]; }
      k.spp[0] = (float)std::max(h[1], h[2]); k.spp[1] = (float)std::max(h[2], h[0]);
      k.spp[2] = (float)std::max(h[0], h[1]);
      k.r0 = 1.f; k.E0 = 0.9f; k.r0pos = 1; k.e0 = 0.9f; k.Ec = 0.f;
      k.Bref[2] = 0.3f; k.g[2] = C.g2;
      k.gamma = 5.f / 3.f; k.gm1 = 2.f / 3.f;
      k.visc = 1; k.rm = 1;
      k.nu1 = C.nu1; k.nu2 = C.nu2; k.nu2dl = (float)(C.nu2 * dlmin); k.nu3 = C.nu3; k.dlmin = (float)dlmin;
      k.dlxy = (float)std::min(h[0], h[1]);
      k.csmag = C.csmag; k.csmag_dl = (float)(C.csmag * dlmin);
      k.nuE = C.nuE; k.nuB = C.nuB; k.c1 = C.c1; k.do_quench = C.quench; k.inv_qmax = 1.f / 8.f; k.qlim = 2.f; k.qeps = 1e-4f;
      k.log_interp = C.log_interp;
      k.inv_tcool = C.tcool > 0 ? 1.f / C.tcool : 0.f; k.e_cool = C.ecool; k.cool_cut = C.cool_cut;
      k.inv_rho_cool = C.cool_cut ? 1.f / C.rhocool : 0.f;
      k.inv_tchromo = C.tchromo > 0 ? 1.f / C.tchromo : 0.f; k.inv_rhobot = C.tchromo > 0 ? 1.f / C.rhobot : 0.f;
      k.corL0 = C.corL0; k.corTu = C.corTu;
      k.d2div = C.d2div; k.d2lim = C.d2lim;
      std::vector<std::vector<float>> d1(F_COUNT, std::vector<float>(g.n)), d4(F_COUNT, std::vector<float>(g.n));
      std::vector<unsigned char> fl1(g.n + 16), fl4(g.n + 16);
      std::vector<std::vector<float>> o1(8, std::vector<float>(g.n)), o4(8, std::vector<float>(g.n));
      float* out1[8];
      float* out4[8];
      for (int c = 0; c < 8; ++c) { out1[c] = o1[c].data(); out4[c] = o4[c].data(); }
      // Each set runs on a uniform mesh and (ZCell types) on a stretched z,
      // dz varying by +-40 %.
      std::vector<float> mesh(4 * nz);
      for (int kz = 0; kz < nz; ++kz) {
        const double th = 2.0 * M_PI / nz;
        const double zc = h[2] * (1.0 + 0.4 * cos(th * (kz + 0.5))), zf = h[2] * (1.0 + 0.4 * cos(th * kz));
        mesh[kz] = (float)zc; mesh[nz + kz] = (float)zf;
        mesh[2 * nz + kz] = (float)(1.0 / zc); mesh[3 * nz + kz] = (float)(1.0 / zf);
      }
      if (stretched) {
        k.hzc = mesh.data(); k.hzf = mesh.data() + nz; k.jzc = mesh.data() + 2 * nz; k.jzf = mesh.data() + 3 * nz;
        rhs<NbZ>(g, k, f, d1, fl1, out1);
        rhs<Nb4Z>(g, k, f, d4, fl4, out4);
        // the mesh must matter: the uniform-mesh right-hand side differs
        std::vector<std::vector<float>> ou(8, std::vector<float>(g.n));
        float* outu[8];
        for (int c = 0; c < 8; ++c) outu[c] = ou[c].data();
        std::vector<std::vector<float>> du(F_COUNT, std::vector<float>(g.n));
        std::vector<unsigned char> flu(g.n + 16);
        rhs<Nb>(g, k, f, du, flu, outu);
        long long changed = 0;
        for (int c = 0; c < 8; ++c)
          for (long long i = 0; i < g.n; ++i) changed += ou[c][i] != o1[c][i];
        if (changed < g.n) {
          printf("stretched mesh left the right-hand side unchanged (%lld values)\n", changed);
          ++bad;
        }
      } else {
        rhs<Nb>(g, k, f, d1, fl1, out1);
        rhs<Nb4>(g, k, f, d4, fl4, out4);
      }
      long long diff = 0, nonfinite = 0;
      for (int c = 0; c < 8; ++c)
        for (long long i = 0; i < g.n; ++i) {
          diff += memcmp(&o1[c][i], &o4[c][i], 4) != 0;
          nonfinite += !std::isfinite(o1[c][i]);
        }
      long long flagged = 0;
      for (long long i = 0; i < g.n; ++i) flagged += fl1[i] != 0;
      printf("case %d%s %dx%dx%d: %lld differing values, %lld non-finite, %lld flagged cells\n", ci,
             stretched ? " stretched" : "", nx, ny, nz, diff, nonfinite, flagged);
      // the second-order switch must take both branches
      bad += diff != 0 || nonfinite != 0 || (C.d2div && (flagged == 0 || flagged == g.n));
    }
  }
  return bad;
}
