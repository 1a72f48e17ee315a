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
// Four-cell threads (Nb4) hold four times the live values of a one-cell
// thread: 2 blocks per SM (128 registers) by default, 3 (80 registers) or 4
// (64) where that measured faster at 512^3.
#ifndef STG_MINB4
#define STG_MINB4 2
#endif
#ifndef STG_MINB4_HI
#define STG_MINB4_HI 3
#endif
#define STG_LB(N, minb) __launch_bounds__(BX * BY * BZ, (N::W == 4 ? STG_MINB4 : (minb)))
#define STG_LB_HI(N, minb) __launch_bounds__(BX * BY * BZ, (N::W == 4 ? STG_MINB4_HI : (minb)))
#define STG_LB_4(N, minb) __launch_bounds__(BX * BY * BZ, (N::W == 4 ? 4 : (minb)))

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

// Four consecutive x-cells of one thread, element-wise arithmetic.  The
// per-cell kernels are templates over the cell type (Nb: one cell, Nb4: four
// cells) and write their arithmetic once on the value type N::T.
struct F4 {
  float v[4];
  F4() = default;
  __device__ __forceinline__ F4(float s) { v[0] = v[1] = v[2] = v[3] = s; }
  __device__ __forceinline__ F4(float a, float b, float c, float d) {
    v[0] = a; v[1] = b; v[2] = c; v[3] = d;
  }
};
#define STG_F4_BIN(op)                                                        \
  __device__ __forceinline__ F4 operator op(const F4& a, const F4& b) {       \
    return F4(a.v[0] op b.v[0], a.v[1] op b.v[1], a.v[2] op b.v[2], a.v[3] op b.v[3]); \
  }
STG_F4_BIN(+)
STG_F4_BIN(-)
STG_F4_BIN(*)
STG_F4_BIN(/)
#undef STG_F4_BIN
__device__ __forceinline__ F4 operator-(const F4& a) { return F4(-a.v[0], -a.v[1], -a.v[2], -a.v[3]); }
__device__ __forceinline__ F4& operator+=(F4& a, const F4& b) { return a = a + b; }
__device__ __forceinline__ F4& operator-=(F4& a, const F4& b) { return a = a - b; }
__device__ __forceinline__ F4& operator*=(F4& a, const F4& b) { return a = a * b; }
// The float versions stay visible next to the F4 overloads below.
using ::expf;
using ::fabsf;
using ::fmaxf;
using ::fminf;
using ::log1pf;
using ::logf;
using ::sqrtf;
using ::cbrtf;
using ::rsqrtf;
#define STG_F4_FN1(fn)                                                        \
  __device__ __forceinline__ F4 fn(const F4& a) {                             \
    return F4(::fn(a.v[0]), ::fn(a.v[1]), ::fn(a.v[2]), ::fn(a.v[3]));        \
  }
#define STG_F4_FN2(fn)                                                        \
  __device__ __forceinline__ F4 fn(const F4& a, const F4& b) {                \
    return F4(::fn(a.v[0], b.v[0]), ::fn(a.v[1], b.v[1]), ::fn(a.v[2], b.v[2]), \
              ::fn(a.v[3], b.v[3]));                                          \
  }
STG_F4_FN1(fabsf)
STG_F4_FN1(sqrtf)
STG_F4_FN1(expf)
STG_F4_FN1(logf)
STG_F4_FN1(log1pf)
STG_F4_FN1(cbrtf)
STG_F4_FN1(rsqrtf)
STG_F4_FN2(fmaxf)
STG_F4_FN2(fminf)
#undef STG_F4_FN1
#undef STG_F4_FN2

// Quotient through the special-function reciprocal (__fdividef, within 2 ulp)
// for divisors that are a density or a quench denominator (>= 1e-30): both
// stay far inside the [2^-126, 2^126] range where that intrinsic is accurate.
#ifndef STG_FASTDIV
#define STG_FASTDIV 1
#endif
__device__ __forceinline__ float fdiv(float a, float b) {
#if STG_FASTDIV
  return __fdividef(a, b);
#else
  return a / b;
#endif
}
__device__ __forceinline__ F4 fdiv(const F4& a, const F4& b) {
  return F4(fdiv(a.v[0], b.v[0]), fdiv(a.v[1], b.v[1]), fdiv(a.v[2], b.v[2]),
            fdiv(a.v[3], b.v[3]));
}

// Periodic neighbour offsets of one cell, offsets -3..3 per axis.
struct Nb {
  using T = float;
  using Base = Nb;
  static constexpr int W = 1;
  int c;
  int kz;       // z index of the cell
  int x[7];
  int y[7];
  int z[7];
  __device__ __forceinline__ int at(int dx, int dy, int dz) const {
    return z[dz + 3] + y[dy + 3] + x[dx + 3];
  }
  __device__ __forceinline__ int ax(int axis, int o) const {
    return axis == 0 ? at(o, 0, 0) : axis == 1 ? at(0, o, 0) : at(0, 0, o);
  }
  __device__ __forceinline__ bool init(const Geo& g);
  // Uniform mesh: the inverse spacings of derivatives whose output sits at a
  // centre (ju) or a face (jd) along axis a, the z diffusion lengths at the
  // centre, the face and a z tap, and the local dl_min (unused when uniform).
  static constexpr bool ZS = false;
  __device__ __forceinline__ bool init(const Geo& g, const KPar&) { return init(g); }
  __device__ __forceinline__ float ju(int a, const KPar& k) const { return k.ih[a]; }
  __device__ __forceinline__ float jd(int a, const KPar& k) const { return k.ih[a]; }
  __device__ __forceinline__ float hzc(const KPar& k) const { return k.sp[2]; }
  __device__ __forceinline__ float hzf(const KPar& k) const { return k.sp[2]; }
  __device__ __forceinline__ float hzc_at(int, const KPar& k) const { return k.sp[2]; }
  __device__ __forceinline__ float dlc(const KPar& k) const { return k.dlmin; }
  // Loads through the read-only path (arrays not written by the launch).
  __device__ __forceinline__ float ld(const float* __restrict__ p) const { return __ldg(p + c); }
  __device__ __forceinline__ float ldat(const float* __restrict__ p, int dx, int dy, int dz) const {
    return __ldg(p + at(dx, dy, dz));
  }
  __device__ __forceinline__ float lda(const float* __restrict__ p, int axis, int o) const {
    return __ldg(p + ax(axis, o));
  }
  // Plain load of the cell's own element of an array the launch rewrites.
  __device__ __forceinline__ float ldw(const float* p) const { return p[c]; }
  // The cell's element of an array of one horizontal plane (nx ny values).
  __device__ __forceinline__ float ldpl(const float* __restrict__ p) const {
    return __ldg(p + (c - z[3]));
  }
  __device__ __forceinline__ void st(float* p, float v) const { p[c] = v; }
  // W consecutive elements at p (element-wise kernels).
  static __device__ __forceinline__ float ldp(const float* __restrict__ p) { return __ldg(p); }
  static __device__ __forceinline__ void stp(float* p, float v) { *p = v; }
  // Per-cell switch flags (one byte per cell, bit a for axis a).
  __device__ __forceinline__ unsigned ldflag(const unsigned char* __restrict__ p) const {
    return __ldg(p + c);
  }
  __device__ __forceinline__ void stflag(unsigned char* p, unsigned f) const {
    p[c] = (unsigned char)f;
  }
  static __device__ __forceinline__ unsigned bits(float v, float lim, int a) {
    return v > lim ? (1u << a) : 0u;
  }
  static __device__ __forceinline__ float sel(unsigned fl, int a, float x, float y) {
    return ((fl >> a) & 1u) ? x : y;
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
  n.kz = k;
  return true;
}
__device__ __forceinline__ bool Nb::init(const Geo& g) { return make_nb(*this, g); }

// Four consecutive x-cells i0..i0+3 (i0 a multiple of 4; requires nx % 4 == 0
// and 16-byte aligned arrays): every tap is one 16-byte load, and the x taps
// are register shifts of the aligned 4-cell chunks left, at and right of i0.
struct Nb4 {
  using T = F4;
  using Base = Nb4;
  static constexpr int W = 4;
  int c;        // offset of cell i0
  int kz;       // z index of the cells
  int x0, xl, xr;   // x of the chunk at, left of and right of i0 (periodic)
  int y[7];
  int z[7];
  __device__ __forceinline__ bool init(const Geo& g) {
    int i = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i >= g.nx || j >= g.ny || k >= g.nz) return false;
    x0 = i;
    xl = wrap(i - 4, g.nx);
    xr = wrap(i + 4, g.nx);
#pragma unroll
    for (int o = -3; o <= 3; ++o) {
      y[o + 3] = wrap(j + o, g.ny) * (int)g.sy;
      z[o + 3] = wrap(k + o, g.nz) * (int)g.sz;
    }
    c = z[3] + y[3] + x0;
    kz = k;
    return true;
  }
  // Uniform mesh: the inverse spacings of derivatives whose output sits at a
  // centre (ju) or a face (jd) along axis a, the z diffusion lengths at the
  // centre, the face and a z tap, and the local dl_min (unused when uniform).
  static constexpr bool ZS = false;
  __device__ __forceinline__ bool init(const Geo& g, const KPar&) { return init(g); }
  __device__ __forceinline__ float ju(int a, const KPar& k) const { return k.ih[a]; }
  __device__ __forceinline__ float jd(int a, const KPar& k) const { return k.ih[a]; }
  __device__ __forceinline__ float hzc(const KPar& k) const { return k.sp[2]; }
  __device__ __forceinline__ float hzf(const KPar& k) const { return k.sp[2]; }
  __device__ __forceinline__ float hzc_at(int, const KPar& k) const { return k.sp[2]; }
  __device__ __forceinline__ float dlc(const KPar& k) const { return k.dlmin; }

  static __device__ __forceinline__ F4 v4(float4 a) { return F4(a.x, a.y, a.z, a.w); }
  static __device__ __forceinline__ F4 row(const float* __restrict__ p, int off) {
    return v4(__ldg(reinterpret_cast<const float4*>(p + off)));
  }
  // Elements s..s+3 of the 8-cell window (a, b), s in 1..3.
  static __device__ __forceinline__ F4 shift(const F4& a, const F4& b, int s) {
    return s == 1 ? F4(a.v[1], a.v[2], a.v[3], b.v[0])
         : s == 2 ? F4(a.v[2], a.v[3], b.v[0], b.v[1])
                  : F4(a.v[3], b.v[0], b.v[1], b.v[2]);
  }
  __device__ __forceinline__ F4 ld(const float* __restrict__ p) const { return row(p, c); }
  __device__ __forceinline__ F4 ldat(const float* __restrict__ p, int dx, int dy, int dz) const {
    const int r = z[dz + 3] + y[dy + 3];
    if (dx == 0) return row(p, r + x0);
    if (dx < 0) return shift(row(p, r + xl), row(p, r + x0), 4 + dx);
    return shift(row(p, r + x0), row(p, r + xr), dx);
  }
  __device__ __forceinline__ F4 lda(const float* __restrict__ p, int axis, int o) const {
    return axis == 0 ? ldat(p, o, 0, 0) : axis == 1 ? ldat(p, 0, o, 0) : ldat(p, 0, 0, o);
  }
  __device__ __forceinline__ F4 ldw(const float* p) const {
    return v4(*reinterpret_cast<const float4*>(p + c));
  }
  __device__ __forceinline__ F4 ldpl(const float* __restrict__ p) const { return row(p, c - z[3]); }
  __device__ __forceinline__ void st(float* p, const F4& v) const { stp(p + c, v); }
  static __device__ __forceinline__ F4 ldp(const float* __restrict__ p) { return row(p, 0); }
  static __device__ __forceinline__ void stp(float* p, const F4& v) {
    *reinterpret_cast<float4*>(p) = make_float4(v.v[0], v.v[1], v.v[2], v.v[3]);
  }
  // Per-cell switch flags: the four cells' bytes as one word (byte l, cell i0+l).
  __device__ __forceinline__ unsigned ldflag(const unsigned char* __restrict__ p) const {
    return __ldg(reinterpret_cast<const unsigned*>(p + c));
  }
  __device__ __forceinline__ void stflag(unsigned char* p, unsigned f) const {
    *reinterpret_cast<unsigned*>(p + c) = f;
  }
  static __device__ __forceinline__ unsigned bits(const F4& v, float lim, int a) {
    return (v.v[0] > lim ? 1u << a : 0u) | (v.v[1] > lim ? 1u << (8 + a) : 0u) |
           (v.v[2] > lim ? 1u << (16 + a) : 0u) | (v.v[3] > lim ? 1u << (24 + a) : 0u);
  }
  static __device__ __forceinline__ F4 sel(unsigned fl, int a, const F4& x, const F4& y) {
    return F4(((fl >> a) & 1u) ? x.v[0] : y.v[0], ((fl >> (8 + a)) & 1u) ? x.v[1] : y.v[1],
              ((fl >> (16 + a)) & 1u) ? x.v[2] : y.v[2], ((fl >> (24 + a)) & 1u) ? x.v[3] : y.v[3]);
  }
};

// A cell type on a stretched z mesh (Sect. Derivatives, reading R19): the
// cell's dz/dk at its centre and lower face, whose inverses are the
// Jacobians of z-derivatives that land there, and its smallest cell size.
template <class B>
struct ZCell : B {
  using Base = B;
  static constexpr bool ZS = true;
  float jc, jf, hc, hf;
  int nzm;
  __device__ __forceinline__ bool init(const Geo& g, const KPar& k) {
    if (!B::init(g)) return false;
    nzm = g.nz;
    hc = __ldg(k.hzc + this->kz);
    hf = __ldg(k.hzf + this->kz);
    jc = __ldg(k.jzc + this->kz);
    jf = __ldg(k.jzf + this->kz);
    return true;
  }
  __device__ __forceinline__ float ju(int a, const KPar& k) const { return a == 2 ? jc : k.ih[a]; }
  __device__ __forceinline__ float jd(int a, const KPar& k) const { return a == 2 ? jf : k.ih[a]; }
  __device__ __forceinline__ float hzc(const KPar&) const { return hc; }
  __device__ __forceinline__ float hzf(const KPar&) const { return hf; }
  __device__ __forceinline__ float hzc_at(int o, const KPar& k) const {
    return o == 0 ? hc : __ldg(k.hzc + wrap(this->kz + o, nzm));
  }
  __device__ __forceinline__ float dlc(const KPar& k) const { return fminf(k.dlxy, hc); }
};
using NbZ = ZCell<Nb>;
using Nb4Z = ZCell<Nb4>;

// eq. (interp) to i+1/2 / i-1/2 and eq. (deriv) to i+1/2 / i-1/2, on a
// functor v(o) giving the operand at offset o along the stencil axis.
template <class V> __device__ __forceinline__ auto s_up(V v) -> decltype(v(0)) {
  return IA_ * (v(0) + v(1)) + IB_ * (v(-1) + v(2)) + IC_ * (v(-2) + v(3));
}
template <class V> __device__ __forceinline__ auto s_dn(V v) -> decltype(v(0)) {
  return IA_ * (v(-1) + v(0)) + IB_ * (v(-2) + v(1)) + IC_ * (v(-3) + v(2));
}
template <class V> __device__ __forceinline__ auto s_du(V v, float ih) -> decltype(v(0)) {
  return (DA_ * (v(1) - v(0)) + DB_ * (v(2) - v(-1)) + DC_ * (v(3) - v(-2))) * ih;
}
template <class V> __device__ __forceinline__ auto s_dd(V v, float ih) -> decltype(v(0)) {
  return (DA_ * (v(0) - v(-1)) + DB_ * (v(1) - v(-2)) + DC_ * (v(2) - v(-3))) * ih;
}

#define LDG(p, i) __ldg((p) + (i))
// Operand functors along one axis of a field at the thread's cell(s).
#define AX(fp, axis) [&](int o) { return n.lda(fp, axis, o); }

template <class T> __device__ __forceinline__ T dens(T t, const KPar& k) {
  if (k.log_interp) return k.r0pos ? k.r0 * expf(t) : expf(t);
  return k.r0 + t;
}

// ----------------------------------------------------------------- lr ------
// ln(rho / r0) = log1p(rho' / r0) of the stored deviation (ln rho if r0 = 0),
// N::W consecutive cells per thread (n a multiple of N::W).
// Also the specific internal energy's deviation e - e0 = (E' + Ec - e0 r') /
// (r' + r0) (Ec = E0 - e0 r0), whose taps the energy fluxes interpolate and
// differentiate; ln rho only when lr is not null (log interpolation).
// With ler (eq. (ediffav)) also ln e - ln <e>_h = log1p((ed - m) / (e0 + m)),
// m = <e - e0>_h the plane mean of the cell's plane (k.emean, sz cells a plane).
template <class N>
__global__ void k_lr_ed(const float* __restrict__ rd, const float* __restrict__ Ed,
                        float* __restrict__ lr, float* __restrict__ ed,
                        float* __restrict__ ler, float* __restrict__ lq, KPar k, long long n,
                        long long sz) {
  using T = typename N::T;
  const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * N::W;
  if (i >= n) return;
  const T r = N::ldp(rd + i);
  if (lr) N::stp(lr + i, k.r0pos ? log1pf(r / k.r0) : logf(r));
  const T Ev = N::ldp(Ed + i);
  const T e = fdiv((Ev + k.Ec) - k.e0 * r, r + k.r0);
  N::stp(ed + i, e);
  if (ler) {
    const float m = (float)k.emean[i / sz];
    N::stp(ler + i, log1pf((e - m) / (k.e0 + m)));
  }
  if (lq) {   // ln(P / P_aver) = ln(E / <E>_h) = log1p((E' - <E'>_h) / (E0 + <E'>_h))
    const long long kz = i / sz;
    N::stp(lq + i, log1pf((Ev - __ldg(k.qm + kz)) / __ldg(k.qden + kz)));
  }
}

// ------------------------------------------------------------- velocity ----
// u_d = p_d / rho_face with rho_face = dens(dn_d ls); the face values dn_d ls
// are also stored (lf, may be null) for the edge densities of the stresses.
template <class N>
__global__ void STG_LB(N, STG_MINB) k_vel(
    const float* __restrict__ ls, const float* __restrict__ px, const float* __restrict__ py,
    const float* __restrict__ pz, float* __restrict__ ux, float* __restrict__ uy,
    float* __restrict__ uz, float* __restrict__ lfx, float* __restrict__ lfy,
    float* __restrict__ lfz, KPar k, Geo g) {
  N n;
  if (!n.init(g, k)) return;
  using T = typename N::T;
  const T lx = s_dn(AX(ls, 0)), ly = s_dn(AX(ls, 1)), lz = s_dn(AX(ls, 2));
  n.st(ux, fdiv(n.ld(px) + k.pref[0], dens(lx, k)));
  n.st(uy, fdiv(n.ld(py) + k.pref[1], dens(ly, k)));
  n.st(uz, fdiv(n.ld(pz) + k.pref[2], dens(lz, k)));
  if (lfx) {
    n.st(lfx, lx);
    n.st(lfy, ly);
    n.st(lfz, lz);
  }
}

// 2D interpolation up along a then b (edge -> centre) of f at the cell.
template <class N>
__device__ __forceinline__ typename N::T up2(const float* __restrict__ f, const N& n, int a, int b) {
  auto inner = [&](int oa) {
    auto v = [&](int ob) {
      int dx = (a == 0 ? oa : 0) + (b == 0 ? ob : 0);
      int dy = (a == 1 ? oa : 0) + (b == 1 ? ob : 0);
      int dz = (a == 2 ? oa : 0) + (b == 2 ? ob : 0);
      return n.ldat(f, dx, dy, dz);
    };
    return s_up(v);
  };
  return s_up(inner);
}

// ---------------------------------------------------------- viscosity ------
// Squared off-diagonal strain on the edges (Smagorinsky runs):
// S_xy^2 (Ez), S_yz^2 (Ex), S_zx^2 (Ey), S_ij = (dd_j u_i + dd_i u_j) / 2.
template <class N>
__global__ void STG_LB(N, STG_MINB) k_strain2(
    const float* __restrict__ ux, const float* __restrict__ uy, const float* __restrict__ uz,
    float* __restrict__ sxy2, float* __restrict__ syz2, float* __restrict__ szx2, KPar k, Geo g) {
  N n;
  if (!n.init(g, k)) return;
  using T = typename N::T;
  T sxy = 0.5f * (s_dd(AX(ux, 1), n.jd(1, k)) + s_dd(AX(uy, 0), n.jd(0, k)));
  T syz = 0.5f * (s_dd(AX(uy, 2), n.jd(2, k)) + s_dd(AX(uz, 1), n.jd(1, k)));
  T szx = 0.5f * (s_dd(AX(uz, 0), n.jd(0, k)) + s_dd(AX(ux, 2), n.jd(2, k)));
  n.st(sxy2, sxy * sxy);
  n.st(syz2, syz * syz);
  n.st(szx2, szx * szx);
}

// -------------------------------------------------------------- Courant ----
// Non-negative maxima kept as the bits of a float: for x >= 0 (and +inf) the
// unsigned order of the bit patterns is the numeric order.  NaN maps to +inf
// (it must win the maximum) and anything below +0, -0 included, to +0.
__device__ __forceinline__ unsigned max_bits(float v) {
  if (!(v == v)) v = INFINITY;
  return __float_as_uint(v > 0.f ? v : 0.f);
}
__device__ __forceinline__ unsigned max_bits(const F4& v) {
  return max(max(max_bits(v.v[0]), max_bits(v.v[1])), max(max_bits(v.v[2]), max_bits(v.v[3])));
}
// |u_perp|^2 = u^2 - (u.B)^2 / B^2, and u^2 where B = 0.
__device__ __forceinline__ float uperp2(float u2, float ub, float B2) {
  return B2 > 0.f ? u2 - ub * ub / B2 : u2;
}
__device__ __forceinline__ F4 uperp2(const F4& u2, const F4& ub, const F4& B2) {
  return F4(uperp2(u2.v[0], ub.v[0], B2.v[0]), uperp2(u2.v[1], ub.v[1], B2.v[1]),
            uperp2(u2.v[2], ub.v[2], B2.v[2]), uperp2(u2.v[3], ub.v[3], B2.v[3]));
}

// Maximum of v over the thread block (NT threads) into *dst (atomic on the
// float bits of max_bits).  Every thread of the block calls it once, at the
// same point.
template <int NT = BX * BY * BZ>
__device__ __forceinline__ void block_max_to(unsigned v, unsigned* dst) {
  __shared__ unsigned sm[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
  if ((tid & 31) == 0) sm[tid >> 5] = v;
  __syncthreads();
  if (tid == 0) {
    unsigned m = 0u;
    for (int w = 0; w < NT / 32; ++w) m = max(m, sm[w]);
    atomicMax(dst, m);
  }
}

// eq. (RMnu): nu1 |u| + nu3 (c_s + c_A) + nu2 dl_min max(0, -div u), centred.
// With CW (the stage whose derivative sets the Courant step) it also reduces
// the wave speed c_s + c_A + |u_perp| of the same centred u and B into *cw.
template <bool SMAG, bool CW, class N>
__device__ __forceinline__ unsigned nu_raw_cell(
    const N& n, const float* __restrict__ ux, const float* __restrict__ uy,
    const float* __restrict__ uz, const float* __restrict__ rd, const float* __restrict__ Ed,
    const float* __restrict__ bx, const float* __restrict__ by, const float* __restrict__ bz,
    const float* __restrict__ sqxy, const float* __restrict__ sqyz,
    const float* __restrict__ sqzx, float* __restrict__ nv, const KPar& k) {
  using T = typename N::T;
  T ucx = s_up(AX(ux, 0)), ucy = s_up(AX(uy, 1)), ucz = s_up(AX(uz, 2));
  const T sxx = s_du(AX(ux, 0), n.ju(0, k)), syy = s_du(AX(uy, 1), n.ju(1, k)),
              szz = s_du(AX(uz, 2), n.ju(2, k));
  T divu = sxx + syy + szz;
  T nu = 0.f;
  const T u2 = ucx * ucx + ucy * ucy + ucz * ucz;
  if (k.nu1 > 0.f) nu = k.nu1 * sqrtf(u2);
  unsigned wbits = 0u;
  if (CW || k.nu3 > 0.f) {
    T bcx = s_up(AX(bx, 0)) + k.Bref[0], bcy = s_up(AX(by, 1)) + k.Bref[1],
          bcz = s_up(AX(bz, 2)) + k.Bref[2];
    T r = n.ld(rd) + k.r0;
    T P = k.gm1 * (n.ld(Ed) + k.E0);
    T cs = sqrtf(k.gamma * P / r);
    T B2 = bcx * bcx + bcy * bcy + bcz * bcz;
    T ca = sqrtf(B2 / r);
    if (k.nu3 > 0.f) nu += k.nu3 * (cs + ca);
    if (CW) {
      const T ub = ucx * bcx + ucy * bcy + ucz * bcz;
      wbits = max_bits(cs + ca + sqrtf(fmaxf(uperp2(u2, ub, B2), T(0.f))));
    }
  }
  // dl_min: of the mesh, or of the cell on a stretched z (R19).
  const float nu2dl = N::ZS ? k.nu2 * n.dlc(k) : k.nu2dl;
  if (k.nu2dl > 0.f) nu += nu2dl * fmaxf(-divu, 0.f);
  if (SMAG) {
    // eq. (nusmag): dl_min Csmag [2 (S_ii^2 - (div u)^2/3 + S_ij^2, i != j)]^1/2.
    T s2 = ((sxx * sxx + syy * syy) + szz * szz) - divu * divu * (1.f / 3.f);
    s2 += 2.f * ((up2(sqxy, n, 0, 1) + up2(sqyz, n, 1, 2)) + up2(sqzx, n, 2, 0));
    nu += (N::ZS ? k.csmag * n.dlc(k) : k.csmag_dl) * sqrtf(2.f * fmaxf(s2, 0.f));
  }
  n.st(nv, nu);
  return wbits;
}

template <bool SMAG, bool CW, class N>
__global__ void __launch_bounds__(BX * BY * BZ, N::W == 4 ? (SMAG ? STG_MINB4 : STG_MINB)
                                                          : (SMAG ? STG_MINB : STG_MINB_HI)) k_nu_raw(
    const float* __restrict__ ux, const float* __restrict__ uy, const float* __restrict__ uz,
    const float* __restrict__ rd, const float* __restrict__ Ed, const float* __restrict__ bx,
    const float* __restrict__ by, const float* __restrict__ bz, const float* __restrict__ sqxy,
    const float* __restrict__ sqyz, const float* __restrict__ sqzx, float* __restrict__ nv,
    unsigned* cw, KPar k, Geo g) {
  N n;
  const bool in = n.init(g, k);
  if constexpr (!CW) {
    if (in) nu_raw_cell<SMAG, false>(n, ux, uy, uz, rd, Ed, bx, by, bz, sqxy, sqyz, sqzx, nv, k);
  } else {
    const unsigned m =
        in ? nu_raw_cell<SMAG, true>(n, ux, uy, uz, rd, Ed, bx, by, bz, sqxy, sqyz, sqzx, nv, k)
           : 0u;
    block_max_to<>(m, cw);
  }
}

// 3-cell max along x, y and z: the maximum over the 3x3x3 neighbourhood.
template <class N>
__global__ void STG_LB(N, STG_MINB) k_nu_max(const float* __restrict__ a,
                                                float* __restrict__ b, Geo g) {
  N n;
  if (!n.init(g)) return;
  using T = typename N::T;
  T m = -INFINITY;
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) m = fmaxf(m, n.ldat(a, dx, dy, dz));
  n.st(b, m);
}

// 3-cell mean along x, y and z (the 3x3x3 mean) and its logarithm.
// With CW (the stage whose derivative sets the Courant step) also the
// maximum of <nu> into *cnu.
template <class N, bool CW>
__global__ void STG_LB(N, STG_MINB_HI) k_nu_smooth(const float* __restrict__ a,
                                                   float* __restrict__ nu,
                                                   float* __restrict__ lnu, unsigned* cnu,
                                                   Geo g) {
  N n;
  const bool in = n.init(g);
  if (!CW && !in) return;
  unsigned m = 0u;
  if (in) {
    using T = typename N::T;
    T sz = 0.f;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
      T sy = 0.f;
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
        T sx = n.ldat(a, -1, dy, dz) + n.ldat(a, 0, dy, dz) + n.ldat(a, 1, dy, dz);
        sy += sx;
      }
      sz += sy;
    }
    T v = sz * (1.f / 27.f);
    n.st(nu, v);
    n.st(lnu, logf(fmaxf(v, 1e-30f)));
    if (CW) m = max_bits(v);
  }
  if constexpr (CW) block_max_to<>(m, cnu);
}

// <nu> = smooth3(max3(nu_raw)) and ln<nu> in one pass that marches along z
// (four-cell threads, nx % 4 == 0, 16-byte aligned arrays).  A thread owns
// the four x-cells i0..i0+3 of row j over NUZ_ZC consecutive planes.  Per raw
// plane it reads rows j-2..j+2 (three 16-byte chunks each) once, and keeps in
// registers the in-plane maxima of the last three planes and the in-plane
// sums of the last three, so each output plane costs one raw plane of loads.
// The maxima are exact and the sums keep k_nu_smooth's order (x, then y,
// then z), so the result equals k_nu_max followed by k_nu_smooth bit for bit.
// With CW also the maximum of <nu> into *cnu (the Courant diffusion limit).
#ifndef NUZ_TY
#define NUZ_TY 4
#endif
#ifndef NUZ_ZC
#define NUZ_ZC 32
#endif
template <bool CW>
__global__ void __launch_bounds__(32 * NUZ_TY) k_nu_maxsmooth(const float* __restrict__ nv,
                                                              float* __restrict__ nu,
                                                              float* __restrict__ lnu,
                                                              unsigned* cnu, Geo g) {
  const int i0 = (blockIdx.x * 32 + threadIdx.x) * 4;
  const int j = blockIdx.y * NUZ_TY + threadIdx.y;
  const int z0 = blockIdx.z * NUZ_ZC;
  const int z1 = min(z0 + NUZ_ZC, g.nz);
  unsigned mb = 0u;
  if (i0 < g.nx && j < g.ny) {
    const int xl = wrap(i0 - 4, g.nx), xr = wrap(i0 + 4, g.nx);
    long long yo[5];
#pragma unroll
    for (int r = 0; r < 5; ++r) yo[r] = (long long)wrap(j + r - 2, g.ny) * g.sy;
    // m[t][r][x]: in-plane 3x3 maxima at planes p-2, p-1, p (t = 0, 1, 2),
    // rows j-1..j+1, x positions i0-1..i0+4.  s[t][l]: in-plane sums of the
    // 3x3 maxima at planes p-3, p-2, p-1 for the four cells.
    float m[3][3][6] = {}, s[3][4] = {};
    for (int p = z0 - 2; p <= z1 + 1; ++p) {
      const long long po = (long long)wrap(p, g.nz) * g.sz;
      float mx[5][6];
#pragma unroll
      for (int r = 0; r < 5; ++r) {
        const float* row = nv + po + yo[r];
        const float4 a = *reinterpret_cast<const float4*>(row + xl);
        const float4 b = *reinterpret_cast<const float4*>(row + i0);
        const float4 c = *reinterpret_cast<const float4*>(row + xr);
        // positions i0-2 .. i0+5
        const float v[8] = {a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y};
#pragma unroll
        for (int x = 0; x < 6; ++x) mx[r][x] = fmaxf(fmaxf(v[x], v[x + 1]), v[x + 2]);
      }
#pragma unroll
      for (int x = 0; x < 6; ++x) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          m[0][r][x] = m[1][r][x];
          m[1][r][x] = m[2][r][x];
          m[2][r][x] = fmaxf(fmaxf(mx[r][x], mx[r + 1][x]), mx[r + 2][x]);
        }
      }
      if (p < z0) continue;
      // Plane p-1: the 3x3x3 maxima, then their sum over x and y.
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        s[0][l] = s[1][l];
        s[1][l] = s[2][l];
        float sy = 0.f;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          float M[3];
#pragma unroll
          for (int d = 0; d < 3; ++d)
            M[d] = fmaxf(fmaxf(m[0][r][l + d], m[1][r][l + d]), m[2][r][l + d]);
          sy += (M[0] + M[1]) + M[2];
        }
        s[2][l] = sy;
      }
      if (p < z0 + 2) continue;
      // Output plane p-2.
      const long long o = (long long)(p - 2) * g.sz + (long long)j * g.sy + i0;
      float4 vv, lv;
      float* vp = &vv.x;
      float* lp = &lv.x;
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const float sz = (s[0][l] + s[1][l]) + s[2][l];
        const float v = sz * (1.f / 27.f);
        vp[l] = v;
        lp[l] = logf(fmaxf(v, 1e-30f));
        if (CW) mb = max(mb, max_bits(v));
      }
      *reinterpret_cast<float4*>(nu + o) = vv;
      *reinterpret_cast<float4*>(lnu + o) = lv;
    }
  }
  if constexpr (CW) block_max_to<32 * NUZ_TY>(mb, cnu);
}

// ln<nu> interpolated to the three faces (first half of the edge values).
template <class N>
__global__ void STG_LB(N, STG_MINB) k_nu_faces(
    const float* __restrict__ lnu, float* __restrict__ lx, float* __restrict__ ly,
    float* __restrict__ lz, Geo g) {
  N n;
  if (!n.init(g)) return;
  using T = typename N::T;
  n.st(lx, s_dn(AX(lnu, 0)));
  n.st(ly, s_dn(AX(lnu, 1)));
  n.st(lz, s_dn(AX(lnu, 2)));
}

// ------------------------------------------------ second-order switch -----
// Bit a of a cell's flag is set where |D2_a ln rho| or |D2_a ln e| exceeds
// d2lim (D2_a f = f(+1) - 2 f + f(-1) along axis a; Sect. Equations,
// do_2nddiv).  The logarithms are those of the stored deviations relative to
// their references, log1p(r'/r0) and log1p(E'/E0) (ln e = ln E - ln rho); the
// constant offsets cancel in D2.
template <class N>
__global__ void STG_LB(N, STG_MINB) k_d2flag(const float* __restrict__ rd,
                                             const float* __restrict__ Ed,
                                             unsigned char* __restrict__ flag, KPar k, Geo g) {
  N n;
  if (!n.init(g, k)) return;
  using T = typename N::T;
  auto lnr = [&](const T& r) { return k.r0pos ? log1pf(r / k.r0) : logf(r); };
  auto lnE = [&](const T& E) { return k.E0 > 0.f ? log1pf(E / k.E0) : logf(E); };
  unsigned fl = 0u;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T lrm = lnr(n.lda(rd, a, -1)), lrc = lnr(n.lda(rd, a, 0)), lrp = lnr(n.lda(rd, a, 1));
    const T lem = lnE(n.lda(Ed, a, -1)) - lrm, lec = lnE(n.lda(Ed, a, 0)) - lrc,
            lep = lnE(n.lda(Ed, a, 1)) - lrp;
    const T d2r = fabsf((lrp - 2.f * lrc) + lrm), d2e = fabsf((lep - 2.f * lec) + lem);
    fl |= N::bits(fmaxf(d2r, d2e), k.d2lim, a);
  }
  n.stflag(flag, fl);
}

// Two-point staggered differences to i+1/2 and i-1/2.
template <class V> __device__ __forceinline__ auto s_du2(V v, float ih) -> decltype(v(0)) {
  return (v(1) - v(0)) * ih;
}
template <class V> __device__ __forceinline__ auto s_dd2(V v, float ih) -> decltype(v(0)) {
  return (v(0) - v(-1)) * ih;
}

// Strain of eq. (itv) from the face velocities: S_xx, S_yy, S_zz at centres
// (strain_diag) and S_xy, S_yz, S_zx on the Ez, Ex, Ey edges (strain_off).
// With the second-order switch compiled in (D2), a derivative along an axis
// whose bit is set in the cell's flags fl is the two-point difference.
template <class T> struct Strain3 { T a, b, c; };
template <bool D2, class N>
__device__ __forceinline__ Strain3<typename N::T> strain_diag(
    const N& n, const float* __restrict__ ux, const float* __restrict__ uy,
    const float* __restrict__ uz, unsigned fl, const KPar& k) {
  Strain3<typename N::T> S{s_du(AX(ux, 0), n.ju(0, k)), s_du(AX(uy, 1), n.ju(1, k)), s_du(AX(uz, 2), n.ju(2, k))};
  if (D2) {
    S.a = N::sel(fl, 0, s_du2(AX(ux, 0), n.ju(0, k)), S.a);
    S.b = N::sel(fl, 1, s_du2(AX(uy, 1), n.ju(1, k)), S.b);
    S.c = N::sel(fl, 2, s_du2(AX(uz, 2), n.ju(2, k)), S.c);
  }
  return S;
}
template <bool D2, class N>
__device__ __forceinline__ Strain3<typename N::T> strain_off(
    const N& n, const float* __restrict__ ux, const float* __restrict__ uy,
    const float* __restrict__ uz, unsigned fl, const KPar& k) {
  using T = typename N::T;
  // (d_a1 f1 + d_a2 f2) / 2, one pair at a time.
  auto pair = [&](const float* f1, int a1, const float* f2, int a2) {
    T d1 = s_dd(AX(f1, a1), n.jd(a1, k)), d2 = s_dd(AX(f2, a2), n.jd(a2, k));
    if (D2) {
      d1 = N::sel(fl, a1, s_dd2(AX(f1, a1), n.jd(a1, k)), d1);
      d2 = N::sel(fl, a2, s_dd2(AX(f2, a2), n.jd(a2, k)), d2);
    }
    return 0.5f * (d1 + d2);
  };
  const T xy = pair(ux, 1, uy, 0);
  const T yz = pair(uy, 2, uz, 1);
  const T zx = pair(uz, 0, ux, 2);
  return Strain3<T>{xy, yz, zx};
}

// -------------------------------------------------------------- stress -----
// Strain, stress (eq. (itv)), J = curl B and eta J on edges, eq. (ohm).
template <class N, bool D2>
__global__ void STG_LB_HI(N, STG_MINB) k_tau(
    const float* __restrict__ ux, const float* __restrict__ uy, const float* __restrict__ uz,
    const float* __restrict__ rd, const float* __restrict__ lfx, const float* __restrict__ lfy,
    const float* __restrict__ lfz, const float* __restrict__ nu, const float* __restrict__ lnx,
    const float* __restrict__ lny, const float* __restrict__ lnz,
    const float* __restrict__ bx, const float* __restrict__ by,
    const float* __restrict__ bz, float* __restrict__ txx, float* __restrict__ tyy,
    float* __restrict__ tzz, float* __restrict__ txy, float* __restrict__ tyz,
    float* __restrict__ tzx, float* __restrict__ Rx, float* __restrict__ Ry,
    float* __restrict__ Rz, float* __restrict__ Jx, float* __restrict__ Jy,
    float* __restrict__ Jz, const unsigned char* __restrict__ flag, KPar k, Geo g) {
  N n;
  if (!n.init(g, k)) return;
  using T = typename N::T;
  T jx = s_dd(AX(bz, 1), n.jd(1, k)) - s_dd(AX(by, 2), n.jd(2, k));
  T jy = s_dd(AX(bx, 2), n.jd(2, k)) - s_dd(AX(bz, 0), n.jd(0, k));
  T jz = s_dd(AX(by, 0), n.jd(0, k)) - s_dd(AX(bx, 1), n.jd(1, k));
  n.st(Jx, jx);
  n.st(Jy, jy);
  n.st(Jz, jz);
  if (!k.visc) return;
  const unsigned fl = D2 ? n.ldflag(flag) : 0u;
  const Strain3<T> Sd = strain_diag<D2>(n, ux, uy, uz, fl, k);
  const T sxx = Sd.a, syy = Sd.b, szz = Sd.c;
  T divu = (sxx + syy) + szz;
  T r = n.ld(rd) + k.r0;
  T nuc = k.rm ? n.ld(nu) : 0.f;
  T nxx = k.rm ? k.sp[0] * nuc : k.nu_const;
  T nyy = k.rm ? k.sp[1] * nuc : k.nu_const;
  T nzz = k.rm ? n.hzc(k) * nuc : k.nu_const;
  n.st(txx, (r * nxx) * (sxx + k.c1 * divu));
  n.st(tyy, (r * nyy) * (syy + k.c1 * divu));
  n.st(tzz, (r * nzz) * (szz + k.c1 * divu));
  // Edge values: the second interpolation of the face values (Ex edge from
  // the y faces along z, Ey from the z faces along x, Ez from the x faces along y).
  // The Ex and Ey edges sit on z faces (their z length at the face, R19).
  const float spp0 = N::ZS ? fmaxf(k.sp[1], n.hzf(k)) : k.spp[0];
  const float spp1 = N::ZS ? fmaxf(n.hzf(k), k.sp[0]) : k.spp[1];
  T nyz = k.rm ? spp0 * expf(s_dn(AX(lny, 2))) : k.nu_const;
  T nzx = k.rm ? spp1 * expf(s_dn(AX(lnz, 0))) : k.nu_const;
  T nxy = k.rm ? k.spp[2] * expf(s_dn(AX(lnx, 1))) : k.nu_const;
  T ryz = dens(s_dn(AX(lfy, 2)), k), rzx = dens(s_dn(AX(lfz, 0)), k),
        rxy = dens(s_dn(AX(lfx, 1)), k);
  const Strain3<T> So = strain_off<D2>(n, ux, uy, uz, fl, k);
  const T sxy = So.a, syz = So.b, szx = So.c;
  n.st(txy, (rxy * nxy) * sxy);
  n.st(tyz, (ryz * nyz) * syz);
  n.st(tzx, (rzx * nzx) * szx);
  n.st(Rx, (k.nuB * nyz) * jx);
  n.st(Ry, (k.nuB * nzx) * jy);
  n.st(Rz, (k.nuB * nxy) * jz);
}

// eq. (quench): T <- T min(max over the axes a0, a1 of max3(q), qlim),
// q = |d2 T| / (M + |d2 T| / qmax), M = |T| + qeps max3|T| along the axis (the
// paper's point value, regularised where it is at roundoff), or max3|T|.
template <bool QM3, class N>
__device__ __forceinline__ typename N::T quench1(const float* __restrict__ f, const N& n, int a0,
                                                 int a1, const KPar& k) {
  using T = typename N::T;
  T fac = -1.f;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    int a = t == 0 ? a0 : a1;
    if (a < 0) continue;
    T v[5], av[5];
#pragma unroll
    for (int o = -2; o <= 2; ++o) {
      v[o + 2] = n.lda(f, a, o);
      av[o + 2] = fabsf(v[o + 2]);
    }
    T m = -1.f;
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      T d2 = (v[o + 2] - 2.f * v[o + 1]) + v[o];
      T a2 = fabsf(d2);
      const T M3 = fmaxf(fmaxf(av[o], av[o + 1]), av[o + 2]);
      const T M = QM3 ? M3 : av[o + 1] + k.qeps * M3;
      T q = fdiv(a2, (M + a2 * k.inv_qmax) + 1e-30f);
      m = fmaxf(m, q);
    }
    fac = fmaxf(fac, m);
  }
  return n.ld(f) * fminf(fac, T(k.qlim));
}

// Quenched stresses, the quenched resistive field eta J (left in the E arrays,
// where k_flux adds -u x B) and the heating densities
// w_c = sum tau_ii S_ii (centre), w_edge = 2 tau_ij S_ij + eta J . J (edge).
// Viscous runs only.
template <class N, bool D2, bool QM3 = false>
__global__ void STG_LB(N, STG_MINB_HI) k_edge(
    const float* __restrict__ txx, const float* __restrict__ tyy, const float* __restrict__ tzz,
    const float* __restrict__ txy, const float* __restrict__ tyz, const float* __restrict__ tzx,
    const float* __restrict__ Rx, const float* __restrict__ Ry, const float* __restrict__ Rz,
    const float* __restrict__ Jx, const float* __restrict__ Jy, const float* __restrict__ Jz,
    const float* __restrict__ ux, const float* __restrict__ uy, const float* __restrict__ uz,
    float* __restrict__ qxx, float* __restrict__ qyy, float* __restrict__ qzz,
    float* __restrict__ qxy, float* __restrict__ qyz, float* __restrict__ qzx,
    float* __restrict__ Ex, float* __restrict__ Ey, float* __restrict__ Ez,
    float* __restrict__ wc, float* __restrict__ wx, float* __restrict__ wy,
    float* __restrict__ wz, const unsigned char* __restrict__ flag, KPar k, Geo g) {
  N n;
  if (!n.init(g, k)) return;
  using T = typename N::T;
  T txx_, tyy_, tzz_, txy_, tyz_, tzx_, rx_, ry_, rz_;
  if (k.do_quench) {
    txx_ = quench1<QM3>(txx, n, 0, -1, k);
    tyy_ = quench1<QM3>(tyy, n, 1, -1, k);
    tzz_ = quench1<QM3>(tzz, n, 2, -1, k);
    txy_ = quench1<QM3>(txy, n, 0, 1, k);
    tyz_ = quench1<QM3>(tyz, n, 1, 2, k);
    tzx_ = quench1<QM3>(tzx, n, 2, 0, k);
    rx_ = quench1<QM3>(Rx, n, 1, 2, k);
    ry_ = quench1<QM3>(Ry, n, 2, 0, k);
    rz_ = quench1<QM3>(Rz, n, 0, 1, k);
    n.st(qxx, txx_);
    n.st(qyy, tyy_);
    n.st(qzz, tzz_);
    n.st(qxy, txy_);
    n.st(qyz, tyz_);
    n.st(qzx, tzx_);
  } else {
    txx_ = n.ld(txx); tyy_ = n.ld(tyy); tzz_ = n.ld(tzz);
    txy_ = n.ld(txy); tyz_ = n.ld(tyz); tzx_ = n.ld(tzx);
    rx_ = n.ld(Rx); ry_ = n.ld(Ry); rz_ = n.ld(Rz);
  }
  n.st(Ex, rx_);
  n.st(Ey, ry_);
  n.st(Ez, rz_);
  const unsigned fl = D2 ? n.ldflag(flag) : 0u;
  const Strain3<T> Sd = strain_diag<D2>(n, ux, uy, uz, fl, k);
  const Strain3<T> So = strain_off<D2>(n, ux, uy, uz, fl, k);
  const T sxx = Sd.a, syy = Sd.b, szz = Sd.c, sxy = So.a, syz = So.b, szx = So.c;
  n.st(wc, (txx_ * sxx + tyy_ * syy) + tzz_ * szz);
  n.st(wx, 2.f * (tyz_ * syz) + rx_ * n.ld(Jx));
  n.st(wy, 2.f * (tzx_ * szx) + ry_ * n.ld(Jy));
  n.st(wz, 2.f * (txy_ * sxy) + rz_ * n.ld(Jz));
}

// ---------------------------------------------------------------- flux -----
struct FluxIn {
  const float *px, *py, *pz, *rd, *Ed, *bx, *by, *bz, *ls, *ux, *uy, *uz;
  const float *qxx, *qyy, *qzz, *qxy, *qyz, *qzx, *Jx, *Jy, *Jz, *nu, *wc, *wx, *wy, *wz;
  const float* ed;   // e - e0 at centres
  const float* ler;  // ln e - ln <e>_h (ediffav)
};
struct FluxOut {
  float *mxx, *myy, *mzz, *mxy, *myx, *mxz, *mzx, *myz, *mzy;
  float *lx1, *lx2, *ly1, *ly2, *lz1, *lz2, *gx, *gy, *gz, *qt;
  float *ex, *ey, *ez;   // in: eta J (viscous runs); out: E = -u x B + eta J
};


// Momentum and induction fluxes: the diagonal and off-diagonal momentum
// fluxes, the Lorentz products and E = -u x B + eta J.
template <class N>
__device__ __forceinline__ void flux_mom_cell(const N& n, const FluxIn& in, const FluxOut& out,
                                              const KPar& k) {
  using T = typename N::T;
  const float* pr[3] = {in.px, in.py, in.pz};
  const float* uu[3] = {in.ux, in.uy, in.uz};
  const float* qd[3] = {in.qxx, in.qyy, in.qzz};
  float* md[3] = {out.mxx, out.myy, out.mzz};
  // With ln(P/P_aver) the pressure gradient is added by k_div instead.
  const T Pd = k.lnpa ? T(0.f) : k.gm1 * n.ld(in.Ed);
  // Diagonal momentum flux at centres: up(p_d) up(u_d) + P - tau_dd.
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float* pp = pr[d];
    const float* up_ = uu[d];
    T v = (s_up(AX(pp, d)) + k.pref[d]) * s_up(AX(up_, d)) + Pd;
    if (k.visc) v -= n.ld(qd[d]);
    n.st(md[d], v);
  }
  // Per edge, the four interpolations of u and B shared by its two
  // off-diagonal momentum fluxes, its two Lorentz products J_a dn(B_b) and
  // E = -u x B (eq. ohm) plus the quenched eta J left by k_edge.  One edge at a
  // time keeps four of the twelve values live.
  const float* B0 = k.Bref;
  // Off-diagonal: p_d carried along axis a, at the (d, a) edge.
  auto off = [&](int d, int a, T ua, const float* tau) {
    const float* pp = pr[d];
    T v = (s_dn(AX(pp, a)) + k.pref[d]) * ua;
    if (k.visc) v -= n.ld(tau);
    return v;
  };
  {  // Ex edge (i, j-1/2, k-1/2)
    const T uy_z = s_dn(AX(in.uy, 2)), uz_y = s_dn(AX(in.uz, 1));
    const T bz_y = s_dn(AX(in.bz, 1)) + B0[2], by_z = s_dn(AX(in.by, 2)) + B0[1];
    n.st(out.myz, off(1, 2, uz_y, in.qyz));
    n.st(out.mzy, off(2, 1, uy_z, in.qyz));
    const T jx = n.ld(in.Jx);
    n.st(out.ly2, jx * bz_y);
    n.st(out.lz1, jx * by_z);
    const T ex = -((uy_z * bz_y) - (uz_y * by_z));
    n.st(out.ex, k.visc ? ex + n.ldw(out.ex) : ex);
  }
  {  // Ey edge (i-1/2, j, k-1/2)
    const T uz_x = s_dn(AX(in.uz, 0)), ux_z = s_dn(AX(in.ux, 2));
    const T bx_z = s_dn(AX(in.bx, 2)) + B0[0], bz_x = s_dn(AX(in.bz, 0)) + B0[2];
    n.st(out.mxz, off(0, 2, uz_x, in.qzx));
    n.st(out.mzx, off(2, 0, ux_z, in.qzx));
    const T jy = n.ld(in.Jy);
    n.st(out.lx1, jy * bz_x);
    n.st(out.lz2, jy * bx_z);
    const T ey = -((uz_x * bx_z) - (ux_z * bz_x));
    n.st(out.ey, k.visc ? ey + n.ldw(out.ey) : ey);
  }
  {  // Ez edge (i-1/2, j-1/2, k)
    const T ux_y = s_dn(AX(in.ux, 1)), uy_x = s_dn(AX(in.uy, 0));
    const T by_x = s_dn(AX(in.by, 0)) + B0[1], bx_y = s_dn(AX(in.bx, 1)) + B0[0];
    n.st(out.mxy, off(0, 1, uy_x, in.qxy));
    n.st(out.myx, off(1, 0, ux_y, in.qxy));
    const T jz = n.ld(in.Jz);
    n.st(out.lx2, jz * by_x);
    n.st(out.ly1, jz * bx_y);
    const T ez = -((ux_y * by_x) - (uy_x * bx_y));
    n.st(out.ez, k.visc ? ez + n.ldw(out.ez) : ez);
  }
}

// Energy fluxes p_d dn(e) - nuE dn(rho nu_dd) dddn(e) at faces, and the
// source -P div u + Q (+ Newtonian cooling).
template <class N>
__device__ __forceinline__ void flux_energy_cell(const N& n, const FluxIn& in,
                                                 const FluxOut& out, const KPar& k) {
  using T = typename N::T;
  const float* pr[3] = {in.px, in.py, in.pz};
  float* go[3] = {out.gx, out.gy, out.gz};
  const float* rd = in.rd;
  const float* Ed = in.Ed;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    // e = e0 + (e - e0): the interpolation weights sum to one.
    auto ed_at = [&](int o) { return n.lda(in.ed, d, o); };
    const T ef = s_dn(ed_at) + k.e0;   // e at the face
    T v = (n.ld(pr[d]) + k.pref[d]) * ef;
    if (k.visc) {
      auto rn_at = [&](int o) {
        const T r = n.lda(rd, d, o) + k.r0;
        const float sp = (N::ZS && d == 2) ? n.hzc_at(o, k) : k.sp[d];
        return r * (k.rm ? sp * n.lda(in.nu, d, o) : T(k.nu_const));
      };
      if (k.ediffav) {   // eq. (ediffav): e dddn(ln e - ln <e>_h)
        auto le_at = [&](int o) { return n.lda(in.ler, d, o); };
        v -= k.nuE * (s_dn(rn_at) * (ef * s_dd(le_at, n.jd(d, k))));
      } else {
        v -= k.nuE * (s_dn(rn_at) * s_dd(ed_at, n.jd(d, k)));
      }
    }
    n.st(go[d], v);
  }
  // -P div u + Q, Q = w_c + up up of the edge heating densities.
  T divu = (s_du(AX(in.ux, 0), n.ju(0, k)) + s_du(AX(in.uy, 1), n.ju(1, k))) +
               s_du(AX(in.uz, 2), n.ju(2, k));
  T P = k.gm1 * (n.ld(Ed) + k.E0);
  T qt = -P * divu;
  if (k.visc) {
    T Q = n.ld(in.wc) + ((up2(in.wz, n, 0, 1) + up2(in.wx, n, 1, 2)) + up2(in.wy, n, 2, 0));
    qt += Q;
  }
  if (k.inv_tcool > 0.f) {
    // Newtonian cooling, eq. (NewtonCool), per volume: -rho (e - e_cool) / t_cool,
    // times the density cutoff of eq. (rhocool).
    const T r = n.ld(in.rd) + k.r0;
    T qn = -((n.ld(Ed) + k.E0) - r * k.e_cool) * k.inv_tcool;
    if (k.cool_cut) {
      const T x = r * k.inv_rho_cool, x2 = x * x;
      qn *= (k.cool_cut == 1 ? x2 : 1.f) / (1.f + x2);
    }
    qt += qn;
  }
  n.st(out.qt, qt);
}

// Two launches with disjoint outputs; they share only the momenta, the
// velocities and E as inputs, and each keeps its live values in registers.
template <class N>
__global__ void STG_LB_HI(N, STG_MINB) k_flux(FluxIn in, FluxOut out, KPar k, Geo g) {
  N n;
  if (!n.init(g, k)) return;
  flux_mom_cell(n, in, out, k);
}

template <class N>
__global__ void STG_LB_HI(N, STG_MINB) k_flux_e(FluxIn in, FluxOut out, KPar k, Geo g) {
  N n;
  if (!n.init(g, k)) return;
  flux_energy_cell(n, in, out, k);
}

// Chromospheric cooling, eq. (ChromoCool), and coronal thin cooling, eq.
// (CoronaCool), added to -P div u + Q after k_flux (runs only when one is on):
//   -rho (rho/rho_bot)^(5/3) (e - <e>)/t_chromo, <e> the plane mean (taken on
//   e - e0 = (E' + Ec - e0 r')/r, where e0 cancels);
//   -L0 T^(-1/2) rho^2 exp(-(T/1e4 K)^2), T = Tunit (gamma - 1) e.
template <class N>
__global__ void STG_LB(N, STG_MINB) k_cool2(const float* __restrict__ rd,
                                            const float* __restrict__ Ed, float* qtp, KPar k,
                                            Geo g) {
  N n;
  if (!n.init(g, k)) return;
  using T = typename N::T;
  const T rdv = n.ld(rd), Edv = n.ld(Ed);
  const T r = rdv + k.r0;
  T qt = n.ldw(qtp);
  if (k.inv_tchromo > 0.f) {
    const T ed = fdiv((Edv + k.Ec) - k.e0 * rdv, r);
    const T x = r * k.inv_rhobot;
    const T x53 = x * cbrtf(x) * cbrtf(x);
    qt -= (r * x53) * ((ed - (float)k.emean[n.kz]) * k.inv_tchromo);
  }
  if (k.corL0 > 0.f) {
    const T Tk = (k.corTu * k.gm1) * fdiv(Edv + k.E0, r);
    const T t4 = Tk * 1e-4f;
    qt -= (k.corL0 * (r * r)) * (expf(-(t4 * t4)) * rsqrtf(Tk));
  }
  n.st(qtp, qt);
}

// ----------------------------------------------------------- divergence ----
struct DivIn {
  const float *px, *py, *pz;
  const float *mxx, *myy, *mzz, *mxy, *myx, *mxz, *mzx, *myz, *mzy;
  const float *lx1, *lx2, *ly1, *ly2, *lz1, *lz2, *gx, *gy, *gz, *qt, *Ex, *Ey, *Ez, *ls;
  const float* f[8];   // stage input (deviations), for the update
  const float* lq;     // ln(P / P_aver) (lnp_aver), else null
  const float* uz;     // face velocity u_z (stellar-atmosphere boundaries)
};

// Pressure gradient along D at the D face through ln(P/P_aver), eq. (pressure):
// exp(dn ln P_aver + dn lq) (dddn lq + dddn ln P_aver), the P_aver factors per
// plane from k_lnpa_tab (the x and y derivatives of ln P_aver vanish).
template <int D, class N>
__device__ __forceinline__ typename N::T lnp_grad(const N& n, const float* lq, const KPar& k) {
  using T = typename N::T;
  auto q = [&](int o) { return n.lda(lq, D, o); };
  const T d = s_dd(q, n.jd(D, k));
  if (D == 2) return (__ldg(k.paz + n.kz) * expf(s_dn(q))) * (d + __ldg(k.dpaz + n.kz));
  return (__ldg(k.pa + n.kz) * expf(s_dn(q))) * d;
}

// F(f) and the RK update: q <- alpha q + F, f_out <- f + beta dt q, for the
// fields in the bit mask M (bit c: field c), each stored as soon as it is
// formed.  mode 0: write F to q only; 1: also update with beta dt = *bdtp.
// Launched as three kernels (momentum; mass and energy; induction), whose
// inputs are disjoint, at 4 blocks per SM: fewer live registers per launch.
// With CR (mass and energy, the stage whose derivative sets the Courant step)
// the launch also reduces max(|dr/dt| / r, |dE/dt| / E) into *cr.
template <class N, int M, bool CR, bool WB = false>
__device__ __forceinline__ unsigned div_cell(const N& n, const DivIn& in, float* const* qs,
                                             float* const* os, float alpha,
                                             const float* bdtp, int mode, const KPar& k) {
  using T = typename N::T;
  const float bdt = mode ? bdtp[0] : 0.f;
  // Rigid (R25) and stellar-atmosphere (R26) z walls (compiled in with WB):
  // the time derivatives of the ghost planes are zero (z faces klo and below
  // are ghosts with R26).
  const bool ghostC = WB && k.wall >= 2 && (n.kz < k.klo || n.kz > k.khi);
  const bool ghostF = k.wall == 3 ? (n.kz <= k.klo || n.kz > k.khi) : ghostC;
  T F0 = 0.f, F4 = 0.f;
  auto fin = [&](int c, const T& Fc) {
    const T F = ((c == 3 || c == 7) ? ghostF : ghostC) ? T(0.f) : Fc;
    if (CR && c == 0) F0 = F;
    if (CR && c == 4) F4 = F;
    const T qq = alpha != 0.f ? alpha * n.ldw(qs[c]) + F : F;
    n.st(qs[c], qq);
    if (mode) n.st(os[c], n.ld(in.f[c]) + bdt * qq);
  };
  // Stellar-atmosphere boundaries (R26): the inflow weight f of the bottom
  // plane's column, from the outward velocity on its inside z face.
  const bool obot = WB && k.wall == 3 && n.kz == k.obot;
  auto open_f = [&]() {
    // constant offsets: a run-time one would put the cell's index tables in local memory
    const T ui = k.osb < 0 ? n.lda(in.uz, 2, 1) : n.lda(in.uz, 2, 0);
    return 1.f / (1.f + expf(ui * ((float)k.osb * k.oinv_u)));
  };
  T Fm = 0.f, Fe = 0.f;
  if (M & 1) {   // eq. (mass)
    const T dxy = s_du(AX(in.px, 0), n.ju(0, k)) + s_du(AX(in.py, 1), n.ju(1, k));
    Fm = -(dxy + s_du(AX(in.pz, 2), n.ju(2, k)));
    if (WB && k.wall == 3 && n.kz == k.otop) {
      // eq. (rbdrylo): the vertical divergence becomes the outward-signed
      // mass flux over the pressure scale height (gamma - 1) e / |g_z|.
      const T r = n.ld(in.f[0]) + k.r0, E = n.ld(in.f[4]) + k.E0;
      const T HP = fdiv(k.gm1 * E, r * k.ogabs);
      Fm = (float)k.ost * fdiv(s_up(AX(in.pz, 2)) + k.pref[2], HP) - dxy;
    }
  }
  if (M & 16)   // eq. (ien)
    Fe = -((s_du(AX(in.gx, 0), n.ju(0, k)) + s_du(AX(in.gy, 1), n.ju(1, k))) + s_du(AX(in.gz, 2), n.ju(2, k))) +
         n.ld(in.qt);
  if ((M & 17) == 17 && obot) {
    // eqs. (rein), (constS) to (addderiv), ideal gas: E relaxes to oE; rho
    // relaxes to orho in inflows (weight f) and takes the isentropic change
    // in outflows.
    const T r = n.ld(in.f[0]) + k.r0, E = n.ld(in.f[4]) + k.E0;
    const T f = open_f();
    const T dE = (k.oE - E) * k.oinv_t;
    Fm = f * ((k.orho - r) * k.oinv_t) +
         (1.f - f) * (Fm + fdiv((dE - Fe) * r, k.gamma * E));
    Fe = dE;
  }
  if (M & 1) fin(0, Fm);
  if (M & 2) {   // eq. (mom), x
    T t = -s_dd(AX(in.mxx, 0), n.jd(0, k));
    t -= s_du(AX(in.mxy, 1), n.ju(1, k));
    t -= s_du(AX(in.mxz, 2), n.ju(2, k));
    t += s_up(AX(in.lx1, 2));
    t -= s_up(AX(in.lx2, 1));
    if (k.g[0] != 0.f) t += dens(s_dn(AX(in.ls, 0)), k) * k.g[0];
    if (k.lnpa) t -= lnp_grad<0>(n, in.lq, k);
    if (obot) t -= open_f() * ((n.ld(in.px) - (float)k.omean[k.klo]) * k.oinv_t);
    fin(1, t);
  }
  if (M & 4) {   // eq. (mom), y
    T t = -s_du(AX(in.myx, 0), n.ju(0, k));
    t -= s_dd(AX(in.myy, 1), n.jd(1, k));
    t -= s_du(AX(in.myz, 2), n.ju(2, k));
    t += s_up(AX(in.ly1, 0));
    t -= s_up(AX(in.ly2, 2));
    if (k.g[1] != 0.f) t += dens(s_dn(AX(in.ls, 1)), k) * k.g[1];
    if (k.lnpa) t -= lnp_grad<1>(n, in.lq, k);
    if (obot) t -= open_f() * ((n.ld(in.py) - (float)k.omean[k.klo + 1]) * k.oinv_t);
    fin(2, t);
  }
  if (M & 8) {   // eq. (mom), z
    T t = -s_du(AX(in.mzx, 0), n.ju(0, k));
    t -= s_du(AX(in.mzy, 1), n.ju(1, k));
    t -= s_dd(AX(in.mzz, 2), n.jd(2, k));
    t += s_up(AX(in.lz1, 1));
    t -= s_up(AX(in.lz2, 0));
    if (k.g[2] != 0.f) t += dens(s_dn(AX(in.ls, 2)), k) * k.g[2];
    if (k.lnpa) t -= lnp_grad<2>(n, in.lq, k);
    fin(3, t);
  }
  if (M & 16) fin(4, Fe);
  // eq. (indu): dB/dt = -curl E
  // R27: the top plane's horizontal field relaxes toward the potential field
  // (targets and plane means from the boundary fill).
  const bool opot = WB && k.wall == 3 && n.kz == k.otop && k.oinv_tpot > 0.f;
  if (M & 32) {
    T t = -(s_du(AX(in.Ez, 1), n.ju(1, k)) - s_du(AX(in.Ey, 2), n.ju(2, k)));
    if (opot) t += (n.ldpl(k.bpx) - (n.ld(in.f[5]) - (float)k.omean[k.klo + 2])) * k.oinv_tpot;
    fin(5, t);
  }
  if (M & 64) {
    T t = -(s_du(AX(in.Ex, 2), n.ju(2, k)) - s_du(AX(in.Ez, 0), n.ju(0, k)));
    if (opot) t += (n.ldpl(k.bpy) - (n.ld(in.f[6]) - (float)k.omean[k.klo + 3])) * k.oinv_tpot;
    fin(6, t);
  }
  if (M & 128) fin(7, -(s_du(AX(in.Ey, 0), n.ju(0, k)) - s_du(AX(in.Ex, 1), n.ju(1, k))));
  if (!CR) return 0u;
  const T r = n.ld(in.f[0]) + k.r0, E = n.ld(in.f[4]) + k.E0;
  return max_bits(fmaxf(fabsf(F0) / r, fabsf(F4) / E));
}

template <class N, int M, bool CR, bool WB = false>
__global__ void STG_LB_4(N, STG_MINB) k_div(DivIn in, float* q0, float* q1, float* q2, float* q3,
                                          float* q4, float* q5, float* q6, float* q7,
                                          float* o0, float* o1, float* o2, float* o3,
                                          float* o4, float* o5, float* o6, float* o7,
                                          float alpha, const float* bdtp,
                                          int mode, unsigned* cr, KPar k, Geo g) {
  N n;
  const bool inside = n.init(g, k);
  float* qs[8] = {q0, q1, q2, q3, q4, q5, q6, q7};
  float* os[8] = {o0, o1, o2, o3, o4, o5, o6, o7};
  if constexpr (!CR) {
    if (inside) div_cell<N, M, false, WB>(n, in, qs, os, alpha, bdtp, mode, k);
  } else {
    const unsigned m = inside ? div_cell<N, M, true>(n, in, qs, os, alpha, bdtp, mode, k) : 0u;
    block_max_to<>(m, cr);
  }
}

// The step dt, and beta_s dt of the three RK stages in FP32 (formed once
// here: a conversion from double runs on the narrow FP64 pipe, so the update
// kernels read the float product instead of forming it per thread).
__device__ __forceinline__ void set_bdt(float* bdt, double dt, float b0, float b1, float b2) {
  bdt[0] = (float)((double)b0 * dt);
  bdt[1] = (float)((double)b1 * dt);
  bdt[2] = (float)((double)b2 * dt);
}
__global__ void k_set_dt(double* dtp, float* bdt, double dt, float b0, float b1, float b2) {
  dtp[0] = dt;
  set_bdt(bdt, dt, b0, b1, b2);
}

// f_out = f + beta dt q for the 8 fields in one launch (blockIdx.y = field),
// 16-byte vectors when every array is 16-byte aligned and n % 4 == 0.
struct Upd8 {
  const float* f[8];
  const float* q[8];
  float* o[8];
};
__global__ void k_update8(Upd8 u, const float* bdtp, long long n, int vec) {
  const int c = blockIdx.y;
  const float bdt = bdtp[0];
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


// -------------------------------------------------------- plane means -----
// Mean over each horizontal plane (constant z) of e - e0 = (E' + Ec - e0 r')/r, in
// FP64 with a fixed summation order: part[k * nb + b] is block b's sum over
// its strided share of plane k; k_plane_final sums the nb parts of a plane.
// PE: the plane sums of E - E0 instead (ln(P/P_aver)).
template <bool PE>
__global__ void k_plane_part(const float* __restrict__ rd, const float* __restrict__ Ed,
                             double* part, KPar k, Geo g) {
  __shared__ double sm[256];
  const int kz = blockIdx.y, nb = gridDim.x;
  const long long m = (long long)g.nx * g.ny;
  const float* r = rd + (long long)kz * g.sz;
  const float* E = Ed + (long long)kz * g.sz;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (long long)nb * blockDim.x)
    acc += PE ? (double)E[i] : (double)(((E[i] + k.Ec) - k.e0 * r[i]) / (r[i] + k.r0));
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(long long)kz * nb + blockIdx.x] = sm[0];
}

__global__ void k_plane_final(const double* part, int nb, double* mean, Geo g) {
  const int kz = blockIdx.x * blockDim.x + threadIdx.x;
  if (kz >= g.nz) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(long long)kz * nb + b];
  mean[kz] = s / ((double)g.nx * g.ny);
}

// ln(P/P_aver), eq. (pressure): one block.  The plane means of E - E0 from
// their nb parts, then per plane k (z periodic over the arrays) P_aver(k) =
// (gamma - 1)(E0 + <E'>_k), and at its lower z face exp(dn_z ln P_aver) and
// dddn_z ln P_aver (eqs. (interp), (deriv) on the nz values of ln P_aver);
// <E'>_k and E0 + <E'>_k as floats for the log ratio of k_lr_ed.
__global__ void k_lnpa_tab(const double* part, int nb, double* mean, float* pa, float* paz,
                           float* dpaz, float* qm, float* qden, KPar k, Geo g) {
  const int nz = g.nz;
  for (int kz = threadIdx.x; kz < nz; kz += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(long long)kz * nb + b];
    mean[kz] = s / ((double)g.nx * g.ny);
  }
  __syncthreads();
  const double a1 = 75.0 / 128.0, b1 = -25.0 / 256.0, c1 = 3.0 / 256.0;   // eq. (interp)
  const double a2 = 75.0 / 64.0, b2 = -25.0 / 384.0, c2 = 3.0 / 640.0;    // eq. (deriv)
  const double gm1 = (double)k.gm1, E0 = (double)k.E0;
  auto lpa = [&](int kz) { return log(gm1 * (E0 + mean[wrap(kz, nz)])); };
  for (int kz = threadIdx.x; kz < nz; kz += blockDim.x) {
    const double l[6] = {lpa(kz - 3), lpa(kz - 2), lpa(kz - 1), lpa(kz), lpa(kz + 1), lpa(kz + 2)};
    pa[kz] = (float)exp(l[3]);
    qm[kz] = (float)mean[kz];
    qden[kz] = (float)(E0 + mean[kz]);
    paz[kz] = (float)exp(a1 * (l[2] + l[3]) + b1 * (l[1] + l[4]) + c1 * (l[0] + l[5]));
    const double jf = k.jzf ? (double)k.jzf[kz] : (double)k.ih[2];
    dpaz[kz] = (float)((a2 * (l[3] - l[2]) + b2 * (l[4] - l[1]) + c2 * (l[5] - l[0])) * jf);
  }
}

// -------------------------------------------------------------- Courant ----
// Per-cell wave speed c_s + c_A + |u_perp|, rate max(|dr/dt|/r, |dE/dt|/E)
// and <nu>; their maxima over the mesh into cmax[0..2] (float bits, atomic).
template <class N>
__global__ void __launch_bounds__(BX * BY * BZ, N::W == 4 ? STG_MINB : STG_MINB_HI) k_courant_part(
    const float* __restrict__ ux, const float* __restrict__ uy, const float* __restrict__ uz,
    const float* __restrict__ rd, const float* __restrict__ Ed, const float* __restrict__ bx,
    const float* __restrict__ by, const float* __restrict__ bz, const float* __restrict__ qr,
    const float* __restrict__ qE, const float* __restrict__ nu, unsigned* cmax, KPar k, Geo g) {
  using T = typename N::T;
  __shared__ unsigned sm[3][BX * BY * BZ / 32];
  N n;
  unsigned m[3] = {0u, 0u, 0u};
  // With closed z walls only the physical centre planes count.
  if (n.init(g, k) && (!k.wall || (n.kz >= k.klo && n.kz <= k.khi))) {
    T ucx = s_up(AX(ux, 0)), ucy = s_up(AX(uy, 1)), ucz = s_up(AX(uz, 2));
    T bcx = s_up(AX(bx, 0)) + k.Bref[0], bcy = s_up(AX(by, 1)) + k.Bref[1],
      bcz = s_up(AX(bz, 2)) + k.Bref[2];
    T r = n.ld(rd) + k.r0;
    T E = n.ld(Ed) + k.E0;
    T cs = sqrtf(k.gamma * (k.gm1 * E) / r);
    T B2 = bcx * bcx + bcy * bcy + bcz * bcz;
    T ca = sqrtf(B2 / r);
    T u2 = ucx * ucx + ucy * ucy + ucz * ucz;
    T ub = ucx * bcx + ucy * bcy + ucz * bcz;
    T w = cs + ca + sqrtf(fmaxf(uperp2(u2, ub, B2), T(0.f)));
    T rate = fmaxf(fabsf(n.ld(qr)) / r, fabsf(n.ld(qE)) / E);
    if (N::ZS) {
      // Stretched z (R19): the limits are minima over cells of the local
      // values, so reduce w / dl and nu / dl (nu_const / dl^2) with dl the
      // cell's smallest size; the final pass then takes dl = 1.
      const float idl = 1.f / n.dlc(k);
      m[0] = max_bits(w * idl);
      m[1] = max_bits(rate);
      if (k.visc) m[2] = max_bits(k.rm ? n.ld(nu) * idl : T(k.nu_const * idl * idl));
    } else {
      m[0] = max_bits(w);
      m[1] = max_bits(rate);
      if (k.visc) m[2] = max_bits(k.rm ? n.ld(nu) : T(k.nu_const));
    }
  }
  const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m[c] = max(m[c], __shfl_xor_sync(0xffffffffu, m[c], o));
  if ((tid & 31) == 0)
    for (int c = 0; c < 3; ++c) sm[c][tid >> 5] = m[c];
  __syncthreads();
  if (tid < 3) {
    unsigned v = 0u;
    for (int wi = 0; wi < BX * BY * BZ / 32; ++wi) v = max(v, sm[tid][wi]);
    atomicMax(cmax + tid, v);
  }
}

// dt = min(Cdt dl/wmax, Cdtr/ratemax, Cdtd dl/(numax f)) in FP64 from the
// three maxima, which it then clears for the next reduction.
__global__ void k_courant_final(unsigned* cmax, double* dt_out, float* bdt, float b0, float b1,
                                float b2, double cdt, double cdtr, double cdtd, double dlmin,
                                double dfac, int nu_is_velocity) {
  if (threadIdx.x != 0) return;
  const double wmax = (double)__uint_as_float(cmax[0]);
  const double rmax = (double)__uint_as_float(cmax[1]);
  const double nmax = (double)__uint_as_float(cmax[2]);
  cmax[0] = cmax[1] = cmax[2] = 0u;
  double tw = wmax > 0 ? cdt * dlmin / wmax : HUGE_VAL;
  double tr = rmax > 0 ? cdtr / rmax : HUGE_VAL;
  double nv = nu_is_velocity ? nmax : nmax / dlmin;
  double td = nv > 0 ? cdtd * dlmin / (nv * dfac) : HUGE_VAL;
  double dt = fmin(tw, fmin(tr, td));
  dt_out[0] = dt;
  set_bdt(bdt, dt, b0, b1, b2);
  dt_out[1] = tw;
  dt_out[2] = tr;
  dt_out[3] = td;
}

// ---------------------------------------------------------- diagnostics ----
// Per-block FP64 partials: sum r', px', py', pz', E', kinetic, magnetic,
// max |div B|, sum (div B)^2, non-finite count.
// On a stretched z (R19) every term is weighted by its cell's z size over the
// mean one (the face spacing for the z-face quantities pz, Bz and their
// energies), the totals the discrete equations conserve.
template <class N>
__global__ void __launch_bounds__(BX * BY * BZ, STG_MINB) k_diag_part(
    const float* __restrict__ rd, const float* __restrict__ px, const float* __restrict__ py,
    const float* __restrict__ pz, const float* __restrict__ Ed, const float* __restrict__ bx,
    const float* __restrict__ by, const float* __restrict__ bz, double* part, KPar k, Geo g) {
  __shared__ double sm[10][BX * BY * BZ];
  N n;
  double v[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
  if (n.init(g, k)) {
    double wc = N::ZS ? (double)n.hzc(k) * k.izbar : 1.0;
    double wf = N::ZS ? (double)n.hzf(k) * k.izbar : 1.0;
    // Closed z walls (R22): the totals the closed box conserves weight the
    // boundary centre planes by one half and count the faces klo+1..khi.
    // Rigid z walls (R25): every plane klo..khi counts once, centres and faces.
    if (k.wall == 1) {
      const int kz = n.kz;
      wc = (kz < k.klo || kz > k.khi) ? 0.0 : (kz == k.klo || kz == k.khi) ? 0.5 : 1.0;
      wf = (kz > k.klo && kz <= k.khi) ? 1.0 : 0.0;
    } else if (k.wall == 2) {
      wc = wf = (n.kz < k.klo || n.kz > k.khi) ? 0.0 : 1.0;
    } else if (k.wall == 3) {   // R26: centres klo..khi, faces klo+1..khi
      wc = (n.kz < k.klo || n.kz > k.khi) ? 0.0 : 1.0;
      wf = (n.kz <= k.klo || n.kz > k.khi) ? 0.0 : 1.0;
    }
    const float* pr[3] = {px, py, pz};
    const float* bb[3] = {bx, by, bz};
    float vals[8] = {LDG(rd, n.c), LDG(px, n.c), LDG(py, n.c), LDG(pz, n.c),
                     LDG(Ed, n.c), LDG(bx, n.c), LDG(by, n.c), LDG(bz, n.c)};
    int bad = 0;
    if (!k.wall || wc > 0.0)
      for (int c = 0; c < 8; ++c) bad += isfinite(vals[c]) ? 0 : 1;
    v[0] = vals[0] * wc;
    v[1] = vals[1] * wc;
    v[2] = vals[2] * wc;
    v[3] = vals[3] * wf;
    v[4] = vals[4] * wc;
    double kin = 0, mag = 0, divb = 0;
    for (int d = 0; d < 3; ++d) {
      auto lsv = [&](int o) {
        float r = LDG(rd, n.ax(d, o));
        if (!k.log_interp) return r;
        return k.r0pos ? log1pf(r / k.r0) : logf(r);
      };
      double rf = (double)dens(s_dn(lsv), k);
      double p = (double)LDG(pr[d], n.c) + k.pref[d];
      const double w = d == 2 ? wf : wc;
      kin += 0.5 * p * p / rf * w;
      double b = (double)LDG(bb[d], n.c) + k.Bref[d];
      mag += 0.5 * b * b * w;
      const float* bp = bb[d];
      divb += (double)s_du(AX(bp, d), n.ju(d, k));
    }
    v[5] = kin;
    v[6] = mag;
    v[7] = (!k.wall || wc > 0.0) ? fabs(divb) : 0.0;
    v[8] = divb * divb * (k.wall ? wc : 1.0);
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

// ------------------------------------------------------- closed z walls ----
// Ghost planes of a box closed at the centre planes lb and ub (reading R22):
// every field is continued across a boundary plane by reflection about it,
// times its parity (r, px, py, E, Bz even; pz, Bx, By odd), repeatedly where
// the box is thinner than the ghost layers.  The plane index m = k - lb of a
// ghost plane is folded into the doubled period P = 2 L, L = ub - lb, as mm:
// centre fields take plane lb + mm (mm <= L) or the reflection lb + P - mm,
// z-face fields (pz, Bz: the face below centre k) face lb + mm (1 <= mm <= L)
// or the reflection lb + P - mm + 1 (mm = 0 read as P).  The odd centred
// fields are zero on the boundary planes themselves.  Every source is a
// physical plane; none is written by this launch except those zeroed odd
// boundary values, which are read as zero.
struct Wall8 {
  float* f[8];
};
__global__ void k_wall_fill(Wall8 w, int lb, int ub, Geo g) {
  const int c = blockIdx.z;
  const int nlo = lb + 1;                      // planes 0..lb, then ub..nz-1
  const int pl = blockIdx.y;
  const int k = pl < nlo ? pl : ub + (pl - nlo);
  const long long m2 = (long long)g.nx * g.ny;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m2 || k >= g.nz) return;
  const bool face = c == 3 || c == 7;
  const bool odd = c == 3 || c == 5 || c == 6;
  const int L = ub - lb, P = 2 * L;
  const int mm = ((k - lb) % P + P) % P;
  float* a = w.f[c];
  if (face) {
    if (k > lb && k <= ub) return;             // a physical face
    // doubled face mm: face lb + mm for 1 <= mm <= L, else the reflection
    const bool dir = mm >= 1 && mm <= L;
    const int src = dir ? lb + mm : lb + P - (mm == 0 ? P : mm) + 1;
    const float v = a[(long long)src * m2 + i];
    a[(long long)k * m2 + i] = (dir || !odd) ? v : -v;
  } else {
    if (k >= lb && k <= ub) {                  // a physical centre plane
      if (odd && (k == lb || k == ub)) a[(long long)k * m2 + i] = 0.f;
      return;
    }
    // doubled centre mm: plane lb + mm for mm <= L, else the reflection
    const bool dir = mm <= L;
    const int src = dir ? lb + mm : lb + P - mm;
    // an odd field is zero on the boundary planes (zeroed by this launch)
    const float v = (odd && (src == lb || src == ub)) ? 0.f : a[(long long)src * m2 + i];
    a[(long long)k * m2 + i] = (dir || !odd) ? v : -v;
  }
}

// Zero the ghost planes of a time derivative (centres outside lb..ub, faces
// outside lb+1..ub).
__global__ void k_wall_zero(Wall8 w, int lb, int ub, Geo g) {
  const int c = blockIdx.z;
  const int nlo = lb + 1;
  const int pl = blockIdx.y;
  const int k = pl < nlo ? pl : ub + (pl - nlo);
  const long long m2 = (long long)g.nx * g.ny;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m2 || k >= g.nz) return;
  const bool face = c == 3 || c == 7;
  const bool ghost = face ? (k <= lb || k > ub) : (k < lb || k > ub);
  if (ghost) w.f[c][(long long)k * m2 + i] = 0.f;
}

// ------------------------------------------------------- rigid z walls ----
// Ghost momenta of a box with rigid walls at the planes lb and ub (reading
// R25): every plane outside lb..ub is a ghost plane, for the face fields too;
// its momentum p_d is set to rho_d u_d(b), the density at the p_d position
// (as k_lr_ed and k_vel form it) times the velocity of the boundary plane b
// (lb below, ub above) at the same (x, y).  The launch reads rho anywhere and
// p_d on the boundary planes, and writes p_d on the ghost planes only.
struct Mom3 {
  float* p[3];
};
// rho at the lower d face of cell (ix, jy, z), formed as k_lr_ed and k_vel form it;
// with log interpolation the logarithms are read from lr (k_lr_ed's output for the
// planes the stencil reaches) when it is given.
__device__ __forceinline__ float rho_face_at(const float* __restrict__ rd,
                                             const float* __restrict__ lr, const KPar& k,
                                             const Geo& g, int d, int ix, int jy, int z) {
  auto ls = [&](int o) {
    const long long c = lin(g, wrap(ix + (d == 0 ? o : 0), g.nx), wrap(jy + (d == 1 ? o : 0), g.ny),
                            wrap(z + (d == 2 ? o : 0), g.nz));
    if (!k.log_interp) return rd[c];
    if (lr) return lr[c];
    return k.r0pos ? log1pf(rd[c] / k.r0) : logf(rd[c]);
  };
  return dens(s_dn(ls), k);
}
__global__ void k_rigid_fill(Mom3 m, const float* __restrict__ rd, const float* __restrict__ lr,
                             KPar k, int lb, int ub, Geo g) {
  const int d = blockIdx.z;
  const int pl = blockIdx.y;                   // planes 0..lb-1, then ub+1..nz-1
  const int kz = pl < lb ? pl : ub + 1 + (pl - lb);
  const long long m2 = (long long)g.nx * g.ny;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m2 || kz >= g.nz) return;
  const int ix = (int)(i % g.nx), jy = (int)(i / g.nx);
  const int b = kz < lb ? lb : ub;
  float* p = m.p[d];
  const float u = fdiv(p[lin(g, ix, jy, b)] + k.pref[d], rho_face_at(rd, lr, k, g, d, ix, jy, b));
  p[lin(g, ix, jy, kz)] = rho_face_at(rd, lr, k, g, d, ix, jy, kz) * u - k.pref[d];
}

// ------------------------------------- stellar-atmosphere z boundaries ----
// Reading R26 (wall 3).  Physical centres klo..khi, z faces klo+1..khi; the
// bottom plane obot (outward direction osb) is the end gravity points to,
// the top otop (ost) the other.  G = klo ghost planes at each end.
//
// k_open_part: row j < G sums, over its plane, the density of the top ghost
// plane otop + ost (j + 1) extrapolated linearly in ln rho from the top plane
// and its inner neighbour; rows G and G + 1 sum the p_x and p_y deviations of
// the bottom plane, rows G + 2 and G + 3 the B_x and B_y deviations of the top
// plane.  k_open_final divides by the plane size.
// ln(rho/r0) (ln rho when r0 = 0) and e - e0 of a cell as k_lr_ed forms them,
// and the density deviation of an extrapolated ln(rho/r0).  FP32 throughout:
// FP64 transcendentals run at a small fraction of the FP32 rate.
__device__ __forceinline__ float open_lnr(float rdv, const KPar& k) {
  return k.r0pos ? log1pf(rdv / k.r0) : logf(rdv);
}
__device__ __forceinline__ float open_ed(float rdv, float Edv, const KPar& k) {
  return fdiv((Edv + k.Ec) - k.e0 * rdv, rdv + k.r0);
}
__device__ __forceinline__ float open_rdev(float l, const KPar& k) {
  return k.r0pos ? k.r0 * expm1f(l) : expf(l);
}
__global__ void k_open_part(const float* __restrict__ rd, const float* __restrict__ px,
                            const float* __restrict__ py, const float* __restrict__ bx,
                            const float* __restrict__ by, double* part, KPar k, Geo g) {
  __shared__ double sm[256];
  const int row = blockIdx.y, nb = gridDim.x, G = k.klo;
  const long long m = (long long)g.nx * g.ny;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (long long)nb * blockDim.x) {
    if (row < G) {
      const float lb_ = open_lnr(rd[(long long)k.otop * m + i], k);
      const float li = open_lnr(rd[(long long)(k.otop - k.ost) * m + i], k);
      acc += (double)(open_rdev(lb_ + (float)(row + 1) * (lb_ - li), k) + k.r0);
    } else if (row < G + 2) {
      acc += (double)(row == G ? px : py)[(long long)k.obot * m + i];
    } else {
      acc += (double)(row == G + 2 ? bx : by)[(long long)k.otop * m + i];
    }
  }
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(long long)row * nb + blockIdx.x] = sm[0];
}
__global__ void k_open_final(const double* part, int nb, int rows, double* mean, Geo g) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(long long)r * nb + b];
  mean[r] = s / ((double)g.nx * g.ny);
}

// Ghost centre planes of rho and E: ln rho and e = E/rho extrapolated
// linearly from the boundary plane b and its inner neighbour; at the top the
// density limited to [orlo, orhi] times its plane mean (omean[j - 1]) and
// e to [e_b / oefac, e_b oefac].  Planes 0..klo-1, then khi+1..nz-1.
__global__ void k_open_fill_c(float* rd, float* Ed, KPar k, Geo g) {
  const int lb = k.klo, ub = k.khi;
  const int pl = blockIdx.y;
  const int kz = pl < lb ? pl : ub + 1 + (pl - lb);
  const long long m2 = (long long)g.nx * g.ny;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m2 || kz >= g.nz) return;
  const bool low = kz < lb;
  const int b = low ? lb : ub, s = low ? -1 : 1, j = low ? lb - kz : kz - ub;
  const float rb = rd[(long long)b * m2 + i], ri = rd[(long long)(b - s) * m2 + i];
  const float eb = open_ed(rb, Ed[(long long)b * m2 + i], k);
  const float ei = open_ed(ri, Ed[(long long)(b - s) * m2 + i], k);
  const float lb_ = open_lnr(rb, k);
  float r = open_rdev(lb_ + (float)j * (lb_ - open_lnr(ri, k)), k);   // deviation
  float e = eb + (float)j * (eb - ei);                                  // e - e0
  if (b == k.otop) {
    const float mj = (float)k.omean[j - 1];
    const float rf = r + k.r0;
    if (rf < k.orlo * mj) r = k.orlo * mj - k.r0;
    if (rf > k.orhi * mj) r = k.orhi * mj - k.r0;
    const float ef = e + k.e0, ebf = eb + k.e0;
    if (ef < ebf / k.oefac) e = ebf / k.oefac - k.e0;
    if (ef > ebf * k.oefac) e = ebf * k.oefac - k.e0;
  }
  rd[(long long)kz * m2 + i] = r;
  // E' = rho (e0 + e') + ... = r' (e0 + e') + r0 e' - Ec
  Ed[(long long)kz * m2 + i] = r * (k.e0 + e) + k.r0 * e - k.Ec;
}

// Ghost momenta and magnetic field, after k_open_fill_c: planes 0..klo (the
// face klo is a ghost face, the centre klo physical), then khi+1..nz-1.
// Bottom: p_x, p_y of centre 2b - kz, p_z of face 2b + 1 - kz (symmetric about
// the boundary point).  Top: rho_d of the filled rho times the boundary
// velocity limited to |u| <= oumax (p_x, p_y from plane b, p_z from the inside
// face).  B_x, B_y extrapolated linearly from b and b - s, B_z from the two
// inside faces; at the bottom B_x, B_y blended toward (oBx, oBy) by f =
// 1/(1 + exp(U oinv_u)), U the outward velocity on the inside face.  Every
// source is a physical plane (nz >= 3 klo + 2); rho is read only.
__global__ void k_open_fill_m(float* px, float* py, float* pz, float* bx, float* by,
                              float* bz, const float* __restrict__ rd,
                              const float* __restrict__ lr, KPar k, Geo g) {
  const int lb = k.klo, ub = k.khi;
  const int pl = blockIdx.y;
  const int kz = pl <= lb ? pl : ub + 1 + (pl - lb - 1);
  const long long m2 = (long long)g.nx * g.ny;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m2 || kz >= g.nz) return;
  const int ix = (int)(i % g.nx), jy = (int)(i / g.nx);
  const bool low = kz <= lb;
  const int b = low ? lb : ub, s = low ? -1 : 1;
  const int mi = low ? lb + 1 : ub;            // the inside face
  const bool centre = low ? kz < lb : true;     // the face kz is a ghost in every case
  const int j = low ? lb - kz : kz - ub;
  const bool top = b == k.otop;
  auto at = [&](int z) { return (long long)z * m2 + i; };
  // outward velocity on the inside face
  const float uzi = fdiv(pz[at(mi)] + k.pref[2], rho_face_at(rd, lr, k, g, 2, ix, jy, mi));
  if (!top) {
    if (centre) {
      px[at(kz)] = px[at(2 * b - kz)];
      py[at(kz)] = py[at(2 * b - kz)];
    }
    pz[at(kz)] = pz[at(2 * b + 1 - kz)];
  } else {
    const float um = k.oumax;
    if (centre) {
      const float ux = fminf(fmaxf(fdiv(px[at(b)] + k.pref[0], rho_face_at(rd, lr, k, g, 0, ix, jy, b)), -um), um);
      const float uy = fminf(fmaxf(fdiv(py[at(b)] + k.pref[1], rho_face_at(rd, lr, k, g, 1, ix, jy, b)), -um), um);
      px[at(kz)] = rho_face_at(rd, lr, k, g, 0, ix, jy, kz) * ux - k.pref[0];
      py[at(kz)] = rho_face_at(rd, lr, k, g, 1, ix, jy, kz) * uy - k.pref[1];
    }
    const float uz = fminf(fmaxf(uzi, -um), um);
    pz[at(kz)] = rho_face_at(rd, lr, k, g, 2, ix, jy, kz) * uz - k.pref[2];
  }
  // magnetic field (stored deviations; the reference cancels in the
  // extrapolation, not in the blend)
  const int d = low ? mi - kz : kz - mi;
  bz[at(kz)] = bz[at(mi)] + (float)d * (bz[at(mi)] - bz[at(mi - s)]);
  if (centre) {
    float vx = bx[at(b)] + (float)j * (bx[at(b)] - bx[at(b - s)]);
    float vy = by[at(b)] + (float)j * (by[at(b)] - by[at(b - s)]);
    if (!top) {
      const float f = 1.f / (1.f + expf((float)s * uzi * k.oinv_u));
      vx = (1.f - f) * vx + f * (k.oBx - k.Bref[0]);
      vy = (1.f - f) * vy + f * (k.oBy - k.Bref[1]);
    }
    bx[at(kz)] = vx;
    by[at(kz)] = vy;
  }
}


#ifdef __CUDACC__   // device-only (dynamic shared memory); not in the host build of the kernels
// ------------------------------------------- top potential field (R27) ----
// Horizontal discrete Fourier transforms of one plane by direct sums along
// one axis at a time (one thread per output element), with twiddles from a
// table of the n roots e^(-2 pi i r / n), the index r = m j advanced modulo n
// (the row kernels keep the table in shared memory: their threads read it at
// scattered places).  k_dft_rows: X[j][m] = sum_i B[j][i] w^(m i);
// k_dft_cols: Y[q][m] = sum_j X[j][m] w^(q j); k_idft_cols2 and k_idft_rows2
// invert two spectra at once, with 1/ny and 1/nx, keeping the real part at the
// end.  FP32 sums of at most a few thousand terms.
__global__ void k_dft_rows(const float* __restrict__ B, float2* X, const float2* __restrict__ w,
                           int nx, int ny) {
  extern __shared__ float2 ws[];
  for (int r = threadIdx.x; r < nx; r += blockDim.x) ws[r] = w[r];
  __syncthreads();
  const int m = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (m >= nx || j >= ny) return;
  const float* b = B + (long long)j * nx;
  float re = 0.f, im = 0.f;
  int r = 0;
  for (int i = 0; i < nx; ++i) {
    const float2 t = ws[r];
    const float v = __ldg(b + i);
    re += v * t.x;
    im += v * t.y;
    r += m;
    if (r >= nx) r -= nx;
  }
  X[(long long)j * nx + m] = make_float2(re, im);
}
__global__ void k_dft_cols(const float2* __restrict__ X, float2* Y, const float2* __restrict__ w,
                           int nx, int ny) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
  if (m >= nx || q >= ny) return;
  float re = 0.f, im = 0.f;
  int r = 0;
  for (int j = 0; j < ny; ++j) {
    const float2 t = __ldg(w + r);
    const float2 v = __ldg(X + (long long)j * nx + m);
    re += v.x * t.x - v.y * t.y;
    im += v.x * t.y + v.y * t.x;
    r += q;
    if (r >= ny) r -= ny;
  }
  Y[(long long)q * nx + m] = make_float2(re, im);
}
__global__ void k_idft_cols2(const float2* __restrict__ P, const float2* __restrict__ Q,
                             float2* ZP, float2* ZQ, const float2* __restrict__ w, int nx,
                             int ny) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (m >= nx || j >= ny) return;
  float pr = 0.f, pi = 0.f, qr = 0.f, qi = 0.f;
  int r = 0;
  for (int q = 0; q < ny; ++q) {
    float2 t = __ldg(w + r);
    t.y = -t.y;                            // e^(+2 pi i q j / ny)
    const float2 a = __ldg(P + (long long)q * nx + m), b = __ldg(Q + (long long)q * nx + m);
    pr += a.x * t.x - a.y * t.y;
    pi += a.x * t.y + a.y * t.x;
    qr += b.x * t.x - b.y * t.y;
    qi += b.x * t.y + b.y * t.x;
    r += j;
    if (r >= ny) r -= ny;
  }
  const float sc = 1.f / (float)ny;
  ZP[(long long)j * nx + m] = make_float2(pr * sc, pi * sc);
  ZQ[(long long)j * nx + m] = make_float2(qr * sc, qi * sc);
}
__global__ void k_idft_rows2(const float2* __restrict__ ZP, const float2* __restrict__ ZQ,
                             float* bp, float* bq, const float2* __restrict__ w, int nx, int ny) {
  extern __shared__ float2 ws[];
  for (int r = threadIdx.x; r < nx; r += blockDim.x) ws[r] = w[r];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= nx || j >= ny) return;
  const float2* zp = ZP + (long long)j * nx;
  const float2* zq = ZQ + (long long)j * nx;
  float p = 0.f, q = 0.f;
  int r = 0;
  for (int m = 0; m < nx; ++m) {
    const float2 t = ws[r];                // Re(z e^(+2 pi i m i / nx)) = z.x t.x + z.y t.y
    const float2 a = __ldg(zp + m), b = __ldg(zq + m);
    p += a.x * t.x + a.y * t.y;
    q += b.x * t.x + b.y * t.y;
    r += i;
    if (r >= nx) r -= nx;
  }
  bp[(long long)j * nx + i] = p / (float)nx;
  bq[(long long)j * nx + i] = q / (float)nx;
}
// The horizontal potential field's spectrum from that of B_z (reading R27):
// P_x = -i s (k_x/|k|) B^_z e^(-i pi m_x/nx) (the x faces half a cell below
// the centres), P_y likewise; no mean or Nyquist part.
__global__ void k_pot_sym(const float2* __restrict__ Y, float2* Px, float2* Py, int nx, int ny,
                          float Lx, float Ly, float s) {
  const int mx = blockIdx.x * blockDim.x + threadIdx.x, my = blockIdx.y;
  if (mx >= nx || my >= ny) return;
  const long long o = (long long)my * nx + mx;
  const int sx = mx < (nx + 1) / 2 ? mx : mx - nx, sy = my < (ny + 1) / 2 ? my : my - ny;
  const bool nyq = ((nx % 2 == 0) && mx == nx / 2) || ((ny % 2 == 0) && my == ny / 2);
  const float kx = 2.f * 3.14159265358979f * (float)sx / Lx, ky = 2.f * 3.14159265358979f * (float)sy / Ly;
  const float kk = sqrtf(kx * kx + ky * ky);
  if (nyq || kk == 0.f) {
    Px[o] = make_float2(0.f, 0.f);
    Py[o] = make_float2(0.f, 0.f);
    return;
  }
  const float2 b = Y[o];
  // -i s c b = s c (b.y, -b.x), then the face phase e^(-i pi m / n)
  float cx, snx, cy, sny;
  sincosf(3.14159265358979f * (float)sx / (float)nx, &snx, &cx);
  sincosf(3.14159265358979f * (float)sy / (float)ny, &sny, &cy);
  const float ax = s * kx / kk, ay = s * ky / kk;
  const float2 qx = make_float2(ax * b.y, -ax * b.x), qy = make_float2(ay * b.y, -ay * b.x);
  Px[o] = make_float2(qx.x * cx + qx.y * snx, qx.y * cx - qx.x * snx);
  Py[o] = make_float2(qy.x * cy + qy.y * sny, qy.y * cy - qy.x * sny);
}

#endif  // __CUDACC__

}  // namespace stg
