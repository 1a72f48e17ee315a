// Op-graph kernels (see graph.cuh): the forward and the hand-written
// transpose (vector-Jacobian) kernel of every primitive, as templates over the
// sweep's precision.  Included by the executor (graph.cu) and by the C ABI
// (api.cu, for the 16-byte access helpers of its RK combinations); plain C++
// apart from the CUDA qualifiers, so that a host build can run them too.
#pragma once

#include <math.h>

#include "graph.cuh"

namespace stg {

// ---------------------------------------------------------------------------
// A cell of a graph launch: 3-D grid of GB x GBY x GBZ thread blocks, so the
// cell's (i, j, k) come from the launch and a periodic neighbour needs no
// division.
// ---------------------------------------------------------------------------
#ifndef GBX
#define GBX 32
#endif
#ifndef GBY
#define GBY 2
#endif
#ifndef GBZ
#define GBZ 4
#endif

struct GCell {
  int i, j, k;
  long long idx;
};

__device__ __forceinline__ bool gcell(GCell& c, const Geo& g) {
  c.i = blockIdx.x * blockDim.x + threadIdx.x;
  c.j = blockIdx.y * blockDim.y + threadIdx.y;
  c.k = blockIdx.z * blockDim.z + threadIdx.z;
  if (c.i >= g.nx || c.j >= g.ny || c.k >= g.nz) return false;
  c.idx = (long long)c.k * g.sz + (long long)c.j * g.sy + c.i;
  return true;
}

// A thread of a graph launch takes GZU cells along z: its first cell from the
// launch, then steps of the launch's z extent (gridDim.z * GBZ).  The
// pointwise and stencil kernels compute every value before they store any,
// so that GZU loads of each operand are in flight together.  One cell per
// thread measured fastest on GB300 (adjoint step at 128^3: 25.3 / 26.5 / 26.7
// / 32.4 ms with 1 / 2 / 4 / 8): the per-op kernels are small enough that
// occupancy, not loads per thread, sets their throughput.
#ifndef GZU
#define GZU 1
#endif

__device__ __forceinline__ GCell gcell_at(const GCell& c0, int u, const Geo& g) {
  GCell c = c0;
  const int dz = u * (int)(gridDim.z * blockDim.z);
  c.k += dz;
  c.idx += (long long)dz * g.sz;
  return c;
}

// A node's constant in the sweep's precision: the FP32 kernels read the
// float copies made when the graph was built (a conversion from double, or
// a double comparison, runs on the FP64 pipe, which is narrow on this GPU).
template <typename T>
__device__ __forceinline__ T kc(double d, float f) {
  if constexpr (sizeof(T) == sizeof(float)) return f;
  else return d;
}

// Periodic neighbour of cell c along an axis (shifted by o).
__device__ __forceinline__ long long nbr(const GCell& c, int axis, int o, const Geo& g) {
  if (axis == 0) return c.idx + (wrap(c.i + o, g.nx) - c.i);
  if (axis == 1) return c.idx + (long long)(wrap(c.j + o, g.ny) - c.j) * g.sy;
  return c.idx + (long long)(wrap(c.k + o, g.nz) - c.k) * g.sz;
}

// The values v(j) at the seven taps c - 3 .. c + 3 along an axis: plain
// strides away from the periodic seam, wrapped indices within 3 cells of it.
template <typename T, class V>
__device__ __forceinline__ void taps7(V v, const GCell& c, int axis, const Geo& g, T t[7]) {
  const long long st = axis == 0 ? 1 : axis == 1 ? g.sy : g.sz;
  const int pos = axis == 0 ? c.i : axis == 1 ? c.j : c.k;
  const int n = axis == 0 ? g.nx : axis == 1 ? g.ny : g.nz;
  if (pos >= 3 && pos + 3 < n) {
#pragma unroll
    for (int o = -3; o <= 3; ++o) t[o + 3] = v(c.idx + o * st);
  } else {
#pragma unroll
    for (int o = -3; o <= 3; ++o) t[o + 3] = v(c.idx + (long long)(wrap(pos + o, n) - pos) * st);
  }
}

// A stencil from the values at its seven taps t[0..6] = c - 3 .. c + 3: up/dn
// are eq. (interp) to i+1/2 and i-1/2; ddup/dddn are eq. (deriv) to i+1/2 and
// i-1/2, divided by the spacing h.
template <typename T>
__device__ __forceinline__ T st_comb(int kind, T h, const T t[7]) {
  const T IA = (T)STG_IA, IB = (T)STG_IB, IC = (T)STG_IC;
  const T DA = (T)STG_DA, DB = (T)STG_DB, DC = (T)STG_DC;
  const T m3 = t[0], m2 = t[1], m1 = t[2], z0 = t[3], p1 = t[4], p2 = t[5], p3 = t[6];
  switch (kind) {
    case ST_UP: return IA * (z0 + p1) + IB * (m1 + p2) + IC * (m2 + p3);
    case ST_DN: return IA * (m1 + z0) + IB * (m2 + p1) + IC * (m3 + p2);
    case ST_DDUP: return (DA * (p1 - z0) + DB * (p2 - m1) + DC * (p3 - m2)) / h;
    default: return (DA * (z0 - m1) + DB * (p1 - m2) + DC * (p2 - m3)) / h;
  }
}

// Stencil value of f at c.
template <typename T>
__device__ __forceinline__ T stencil_at(const T* f, const GCell& c, int axis, int kind, T h,
                                        const Geo& g) {
  T t[7];
  taps7<T>([&](long long j) { return f[j]; }, c, axis, g, t);
  return st_comb(kind, h, t);
}

// The same stencil of the values v(idx) of a functor at the taps.
template <typename T, class V>
__device__ __forceinline__ T stencil_fn(V v, const GCell& c, int axis, int kind, T h,
                                        const Geo& g) {
  T t[7];
  taps7<T>(v, c, axis, g, t);
  return st_comb(kind, h, t);
}
// Transposed kind and sign of a stencil: up^T = dn, dn^T = up, ddup^T =
// -dddn, dddn^T = -ddup (periodic summation by parts).
__device__ __forceinline__ int st_transpose(int kind) {
  return kind == ST_UP ? ST_DN : kind == ST_DN ? ST_UP : kind == ST_DDUP ? ST_DDDN : ST_DDUP;
}
__device__ __forceinline__ bool st_negates(int kind) { return kind == ST_DDUP || kind == ST_DDDN; }

// ---------------------------------------------------------------------------
// Quench, eq. (quench) with reading R8, as one node: out = T min(fac, qlim),
// fac = the max over the node's axes of max3 along the axis of
// q = |D2 T| / ((M + |D2 T| / qmax) + 1e-30), D2 T = T(+1) - 2 T + T(-1) and
// M = |T| + eps max3 |T| (eps = c2 >= 0), or M = max3 |T| (c2 < 0).  Its
// transpose follows the rules of the primitive nodes it stands for: a max
// splits the gradient evenly on a tie (pairwise, the inner pair first),
// |x|' = sign x with sign 0 = 0, the clamp passes the gradient where
// fac <= qlim.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void max_w(T a, T b, T& wa, T& wb) {
  wa = a > b ? (T)1 : (a == b ? (T)0.5 : (T)0);
  wb = b > a ? (T)1 : (a == b ? (T)0.5 : (T)0);
}
template <typename T>
__device__ __forceinline__ T sgn(T a) {
  return a > (T)0 ? (T)1 : (a < (T)0 ? (T)-1 : (T)0);
}

// The quench's divisions: the fast intrinsic in FP32 (within 2 ulp; the
// divisors are >= 1e-30 and far below 2^126), IEEE division in FP64.
template <typename T>
__device__ __forceinline__ T qdiv(T a, T b) {
  if constexpr (sizeof(T) == sizeof(float)) return __fdividef(a, b);
  else return a / b;
}

// q at z = c + s e_ax from T at z - 1, z, z + 1 (vm, v0, vp), and (dq) its
// derivatives with respect to those (through D2 T and through M).
template <typename T>
__device__ __forceinline__ T q_val(T vm, T v0, T vp, T iq, T eps, T* dq) {
  const T d2 = (vp - (T)2 * v0) + vm, a2 = fabs(d2);
  const T am = fabs(vm), a0 = fabs(v0), ap = fabs(vp);
  const T inner = am >= a0 ? am : a0;
  const T M3 = inner >= ap ? inner : ap;
  // M = cM max3|T| + cP |T|.
  const T cM = eps < (T)0 ? (T)1 : eps, cP = eps < (T)0 ? (T)0 : (T)1;
  const T M = eps < (T)0 ? M3 : a0 + eps * M3;
  const T den = (M + a2 * iq) + (T)1e-30;
  const T q = qdiv(a2, den);
  if (dq) {
    T wim, wi0, woi, wop;
    max_w(am, a0, wim, wi0);
    max_w(inner, ap, woi, wop);
    // a2 / den^2 as q / den: den^2 underflows in FP32 where T and D2 T are
    // both zero (den = 1e-30), and 0 / 0 would poison the cotangent.
    const T qd = qdiv(q, den);
    const T dq_da2 = qdiv((T)1, den) - iq * qd;
    const T dq_dM = -qd;
    const T sd = sgn(d2);
    dq[0] = dq_da2 * sd + dq_dM * (cM * (woi * wim)) * sgn(vm);
    dq[1] = dq_da2 * sd * (T)-2 + dq_dM * (cM * (woi * wi0) + cP) * sgn(v0);
    dq[2] = dq_da2 * sd + dq_dM * (cM * wop) * sgn(vp);
  }
  return q;
}
template <typename T>
__device__ __forceinline__ T q_at(const T* A, const GCell& c, int ax, int s, T iq, T eps,
                                  const Geo& g, T* dq) {
  return q_val(A[nbr(c, ax, s - 1, g)], A[nbr(c, ax, s, g)], A[nbr(c, ax, s + 1, g)], iq, eps,
               dq);
}

// fac at c, and (when wq) the weights of the three q of each axis in fac:
// wq[3 t + p + 1] for axis t and position p.  qf(t, ax, s) is q at
// c + s e_ax (axis slot t): formed from T, or read from the transpose's
// per-cell q arrays.
template <typename T, class QF>
__device__ __forceinline__ T quench_fac(QF qf, int a0, int a1, T* wq) {
  T m[2] = {0, 0}, w[2][3];
  for (int t = 0; t < 2; ++t) {
    const int ax = t == 0 ? a0 : a1;
    if (ax < 0) continue;
    const T qm = qf(t, ax, -1), q0 = qf(t, ax, 0), qp = qf(t, ax, 1);
    const T inner = qm >= q0 ? qm : q0;
    m[t] = inner >= qp ? inner : qp;
    T wim, wi0, woi, wop;
    max_w(qm, q0, wim, wi0);
    max_w(inner, qp, woi, wop);
    w[t][0] = woi * wim;
    w[t][1] = woi * wi0;
    w[t][2] = wop;
  }
  T fac = m[0], wf0 = 1, wf1 = 0;
  if (a1 >= 0) {
    fac = m[0] >= m[1] ? m[0] : m[1];
    max_w(m[0], m[1], wf0, wf1);
  }
  if (wq)
    for (int p = 0; p < 3; ++p) {
      wq[p] = wf0 * w[0][p];
      wq[3 + p] = a1 >= 0 ? wf1 * w[1][p] : (T)0;
    }
  return fac;
}

// Transpose, q pass (per cell z, per axis slot t): q(z) and its derivatives
// with respect to T at z - 1, z, z + 1, into Q[(4 t + 0 .. 3) n + z], formed
// once here instead of at every tap of the two passes that follow.
template <typename T>
__global__ void g_quench_q(GNode nd, const T* A, T* Q, Geo g) {
  GCell c0;
  if (!gcell(c0, g)) return;
  const T iq = (T)1 / kc<T>(nd.c0, nd.f0), eps = kc<T>(nd.c2, nd.f2);
  for (int u = 0; u < GZU; ++u) {
    const GCell c = gcell_at(c0, u, g);
    if (c.k >= g.nz) break;
    for (int t = 0; t < 2; ++t) {
      const int ax = t == 0 ? nd.axis : nd.sk;
      if (ax < 0) continue;
      T dq[3];
      const T q = q_at(A, c, ax, 0, iq, eps, g, dq);
      Q[(long long)(4 * t) * g.n + c.idx] = q;
      for (int k = 0; k < 3; ++k) Q[(long long)(4 * t + 1 + k) * g.n + c.idx] = dq[k];
    }
  }
}

// Transpose, first pass (per output cell y): S0 = gbar C (the product's own
// term) and S[1 + 3 t + p + 1] = gbar T dC/dfac dfac/dq, the cotangent each
// q of axis t at position p receives from y.
template <typename T>
__global__ void g_quench_b1(GNode nd, const T* A, const T* Q, const T* gout, T* S, Geo g) {
  GCell c0;
  if (!gcell(c0, g)) return;
  const T qlim = kc<T>(nd.c1, nd.f1);
  for (int u = 0; u < GZU; ++u) {
    const GCell c = gcell_at(c0, u, g);
    if (c.k >= g.nz) break;
    T wq[6];
    const T fac = quench_fac<T>(
        [&](int t, int ax, int s) { return Q[(long long)(4 * t) * g.n + nbr(c, ax, s, g)]; },
        nd.axis, nd.sk, wq);
    const T gg = gout[c.idx];
    const T C = fac > qlim ? qlim : fac;
    const T dC = fac <= qlim ? (T)1 : (T)0;
    const T base = gg * A[c.idx] * dC;
    S[c.idx] = gg * C;
    for (int j = 0; j < 6; ++j) S[(long long)(1 + j) * g.n + c.idx] = base * wq[j];
  }
}

// Transpose, second pass (per input cell x): Tbar(x) = S0(x) + the sum over
// the axes and the three q positions z = x + r e_a whose stencils hold x of
// qbar(z) dq(z)/dT(x), qbar(z) = sum_p S[.. p](z - p e_a).
template <typename T>
__global__ void g_quench_b3(GNode nd, const T* Q, const T* S, T* gA, int wA, Geo g) {
  GCell c0;
  if (!gcell(c0, g)) return;
  for (int u = 0; u < GZU; ++u) {
    const GCell c = gcell_at(c0, u, g);
    if (c.k >= g.nz) break;
    T acc = S[c.idx];
    for (int t = 0; t < 2; ++t) {
      const int ax = t == 0 ? nd.axis : nd.sk;
      if (ax < 0) continue;
      for (int r = -1; r <= 1; ++r) {
        T qbar = 0;
        for (int p = -1; p <= 1; ++p)
          qbar += S[(long long)(1 + 3 * t + p + 1) * g.n + nbr(c, ax, r - p, g)];
        // d q(z) / d T(x), z = x + r e_ax: the derivative at z's tap 1 - r.
        acc += qbar * Q[(long long)(4 * t + 2 - r) * g.n + nbr(c, ax, r, g)];
      }
    }
    gA[c.idx] = wA ? acc : gA[c.idx] + acc;
  }
}

// Quench forward (G_QUENCH): out = T min(fac, qlim).
template <typename T>
__global__ void g_quench_f(GNode nd, const T* A, T* out, Geo g) {
  GCell c0;
  if (!gcell(c0, g)) return;
  for (int u = 0; u < GZU; ++u) {
    const GCell c = gcell_at(c0, u, g);
    if (c.k >= g.nz) break;
    const T iq = (T)1 / kc<T>(nd.c0, nd.f0), qlim = kc<T>(nd.c1, nd.f1);
    const T eps = kc<T>(nd.c2, nd.f2);
    const T fac = quench_fac<T>(
        [&](int, int ax, int s) { return q_at(A, c, ax, s, iq, eps, g, (T*)nullptr); }, nd.axis,
        nd.sk, (T*)nullptr);
    out[c.idx] = A[c.idx] * (fac > qlim ? qlim : fac);
  }
}

// y = st (op) b of a G_STBIN node (side 1: b first).
template <typename T>
__device__ __forceinline__ T stbin_val(const GNode& nd, T st, T b) {
  if (nd.iop == G_MUL) return st * b;
  if (nd.iop == G_ADD) return nd.side ? b + st : st + b;
  return nd.side ? b - st : st - b;     // G_SUB
}

template <typename T>
__device__ __forceinline__ T fwd_value(int op, const GNode& nd, const T* A, const T* B,
                                       const T* mesh, const GCell& c, const Geo& g) {
  const long long idx = c.idx;
  switch (op) {
    case G_STENCIL: return stencil_at(A, c, nd.axis, nd.sk, kc<T>(nd.c0, nd.f0), g);
    case G_STBIN:
      return stbin_val(nd, stencil_at(A, c, nd.axis, nd.sk, kc<T>(nd.c0, nd.f0), g), B[idx]);
    case G_STMUL:
      return stencil_fn<T>([&](long long j) { return A[j] * B[j]; }, c, nd.axis, nd.sk,
                           kc<T>(nd.c0, nd.f0), g);
    case G_STEXP: return exp(stencil_at(A, c, nd.axis, nd.sk, kc<T>(nd.c0, nd.f0), g));
    case G_NB3: {
      const T m = A[nbr(c, nd.axis, nd.sk, g)], z = A[idx], p = A[nbr(c, nd.axis, -nd.sk, g)];
      if (nd.iop == G_ADD) return (m + z) + p;
      const T in = m >= z ? m : z;
      return in >= p ? in : p;
    }
    case G_ST2: {
      const T s1 = stencil_at(A, c, nd.axis, nd.sk, kc<T>(nd.c0, nd.f0), g);
      const T s2 = stencil_at(B, c, nd.axis2, nd.sk2, kc<T>(nd.h2, nd.fh2), g);
      return nd.iop == G_ADD ? s1 + s2 : s1 - s2;
    }
    case G_SHIFT: return A[nbr(c, nd.axis, nd.sk, g)];
    default: return mesh[(long long)nd.sk * g.nz + c.k];   // G_ZFIELD
  }
}

// The ops whose value at a cell reads only that cell of their operands: they
// run as flat kernels over the arrays (g_forward_pw, g_backward_pw).
__host__ __device__ __forceinline__ bool pointwise_op(int op) {
  return op == G_ADD || op == G_SUB || op == G_MUL || op == G_DIV || op == G_MAX ||
         op == G_EXP || op == G_LOG || op == G_LOG1P || op == G_SQRT || op == G_ABS ||
         op == G_AXPB || op == G_CLAMPMIN || op == G_CLAMPMAX || op == G_STEP || op == G_CONST;
}

// A pointwise op's value from its operands' values a, b at the cell.
template <typename T>
__device__ __forceinline__ T pw_value(int op, const GNode& nd, T a, T b) {
  switch (op) {
    case G_ADD: return a + b;
    case G_SUB: return a - b;
    case G_MUL: return a * b;
    case G_DIV: return a / b;
    case G_MAX: return a >= b ? a : b;
    case G_EXP: return exp(a);
    case G_LOG: return log(a);
    case G_LOG1P: return log1p(a);
    case G_SQRT: return sqrt(a);
    case G_ABS: return fabs(a);
    case G_AXPB: return kc<T>(nd.c0, nd.f0) * a + kc<T>(nd.c1, nd.f1);
    case G_CLAMPMIN: return a < kc<T>(nd.c0, nd.f0) ? kc<T>(nd.c0, nd.f0) : a;
    case G_CLAMPMAX: return a > kc<T>(nd.c0, nd.f0) ? kc<T>(nd.c0, nd.f0) : a;
    case G_STEP: return a > kc<T>(nd.c0, nd.f0) ? (T)1 : (T)0;
    default: return kc<T>(nd.c0, nd.f0);  // G_CONST
  }
}

// The folded sum and the epilogue of a node's value v (C's value cv).
template <typename T>
__device__ __forceinline__ T finish(const GNode& nd, T v, T cv) {
  if (nd.pop) v = nd.pop == 1 ? v + cv : nd.pop == 2 ? v - cv : cv - v;
  return nd.ep ? kc<T>(nd.ps, nd.fps) * v + kc<T>(nd.pt, nd.fpt) : v;
}

// Four consecutive elements i .. i + 3 as 16-byte loads and stores (i a
// multiple of 4, the array 16-byte aligned).
template <typename T>
__device__ __forceinline__ void ld4(const T* p, long long i, T (&v)[4]) {
  if constexpr (sizeof(T) == sizeof(float)) {
    const float4 x = *reinterpret_cast<const float4*>(p + i);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  } else {
    const double2 x = *reinterpret_cast<const double2*>(p + i);
    const double2 y = *reinterpret_cast<const double2*>(p + i + 2);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
  }
}
template <typename T>
__device__ __forceinline__ void st4(T* p, long long i, const T (&v)[4]) {
  if constexpr (sizeof(T) == sizeof(float)) {
    *reinterpret_cast<float4*>(p + i) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    *reinterpret_cast<double2*>(p + i) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + i + 2) = make_double2(v[2], v[3]);
  }
}

// Pointwise forward over n cells: with vec (every array 16-byte aligned and n
// a multiple of 4) four cells a thread through 16-byte accesses, which keeps
// enough bytes in flight per SM; else one cell at a time.  Grid-stride.
template <typename T, int OP>
__global__ void g_forward_pw(GNode nd, const T* A, const T* B, const T* C, T* out, long long n,
                             int vec) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (vec) {
    for (; t < n / 4; t += stride) {
      const long long i = 4 * t;
      T a[4] = {0, 0, 0, 0}, b[4] = {0, 0, 0, 0}, cv[4] = {0, 0, 0, 0}, r[4];
      if (A) ld4(A, i, a);
      if (B) ld4(B, i, b);
      if (nd.pop) ld4(C, i, cv);
#pragma unroll
      for (int k = 0; k < 4; ++k) r[k] = finish(nd, pw_value(OP, nd, a[k], b[k]), cv[k]);
      st4(out, i, r);
    }
  } else {
    for (; t < n; t += stride) {
      const T a = A ? A[t] : (T)0, b = B ? B[t] : (T)0, cv = nd.pop ? C[t] : (T)0;
      out[t] = finish(nd, pw_value(OP, nd, a, b), cv);
    }
  }
}

// Every node but the pointwise ones, G_QUENCH (g_quench_f) and G_PMEAN; one
// instance per op.
template <typename T, int OP>
__global__ void g_forward(GNode nd, const T* A, const T* B, const T* C, T* out, const T* mesh,
                          Geo g) {
  GCell c0;
  if (!gcell(c0, g)) return;
  T r[GZU];
#pragma unroll
  for (int u = 0; u < GZU; ++u) {
    const GCell c = gcell_at(c0, u, g);
    if (c.k < g.nz)
      r[u] = finish(nd, fwd_value(OP, nd, A, B, mesh, c, g), nd.pop ? C[c.idx] : (T)0);
  }
#pragma unroll
  for (int u = 0; u < GZU; ++u) {
    const GCell c = gcell_at(c0, u, g);
    if (c.k < g.nz) out[c.idx] = r[u];
  }
}

// Transpose kernels.  Pointwise rules follow the usual subgradient choices:
// |x|' = sign(x) with sign(0) = 0; clamp passes the gradient where the bound
// holds with equality; max(a, b) splits it evenly on ties.
template <typename T>
__device__ __forceinline__ void bwd_value(int op, const GNode& nd, const T* A, const T* B,
                                          const T* out, const T* gout, const GCell& c,
                                          const Geo& g, T& ca, T& cb) {
  const long long idx = c.idx;
  ca = 0;
  cb = 0;
  if (op == G_STENCIL) {
    // Gather form of the transpose: up^T = dn, dn^T = up, ddup^T = -dddn,
    // dddn^T = -ddup (periodic summation by parts).
    int kind = nd.sk;
    T v = stencil_at(gout, c, nd.axis, st_transpose(kind), kc<T>(nd.c0, nd.f0), g);
    ca = st_negates(kind) ? -v : v;
  } else if (op == G_STBIN) {
    // y = st(a) (op) b: the stencil's transpose of the cotangent of st(a),
    // which is g (add), -+g (sub) or g b (mul) at each tap.
    const int tk = st_transpose(nd.sk);
    const T sg = st_negates(nd.sk) ? (T)-1 : (T)1;
    const T gg = gout[idx];
    if (nd.iop == G_MUL) {
      ca = sg * stencil_fn<T>([&](long long j) { return gout[j] * B[j]; }, c, nd.axis, tk,
                              kc<T>(nd.c0, nd.f0), g);
      cb = gg * stencil_at(A, c, nd.axis, nd.sk, kc<T>(nd.c0, nd.f0), g);
    } else {
      const T v = sg * stencil_at(gout, c, nd.axis, tk, kc<T>(nd.c0, nd.f0), g);
      const bool neg_st = nd.iop == G_SUB && nd.side;    // b - st
      const bool neg_b = nd.iop == G_SUB && !nd.side;    // st - b
      ca = neg_st ? -v : v;
      cb = neg_b ? -gg : gg;
    }
  } else if (op == G_STMUL) {
    // y = st(a b): the transposed stencil of g, times the other factor.
    T v = stencil_at(gout, c, nd.axis, st_transpose(nd.sk), kc<T>(nd.c0, nd.f0), g);
    if (st_negates(nd.sk)) v = -v;
    ca = v * B[idx];
    cb = v * A[idx];
  } else if (op == G_STEXP) {
    // y = ps exp(st(a)) + pt: the stencil's transpose of g (y - pt), the
    // epilogue's factor included (it is in y).
    const T pt = kc<T>(nd.pt, nd.fpt);
    T v = stencil_fn<T>([&](long long j) { return gout[j] * (out[j] - pt); }, c, nd.axis,
                        st_transpose(nd.sk), kc<T>(nd.c0, nd.f0), g);
    ca = st_negates(nd.sk) ? -v : v;
  } else if (op == G_NB3) {
    // Gather over the three outputs y = x - o, x, x + o (o = sk) that read x
    // as their a(y + o), a(y), a(y - o); a max passes g by the primitive
    // nodes' rule (an even split on a tie, the inner pair first).
    const int ax = nd.axis, o = nd.sk;
    const T gm = gout[nbr(c, ax, -o, g)], g0 = gout[idx], gp = gout[nbr(c, ax, o, g)];
    if (nd.iop == G_ADD) {
      ca = (gm + g0) + gp;
    } else {
      const T a0 = A[idx], am = A[nbr(c, ax, -o, g)], am2 = A[nbr(c, ax, -2 * o, g)];
      const T ap = A[nbr(c, ax, o, g)], ap2 = A[nbr(c, ax, 2 * o, g)];
      T wm, wz, wi, wp;
      max_w(a0, am, wm, wz);   // y = x - o: (a0 op am) op am2, x in the inner first slot
      max_w(a0 >= am ? a0 : am, am2, wi, wp);
      T acc = gm * (wi * wm);
      max_w(ap, a0, wm, wz);   // y = x: (ap op a0) op am, x in the inner second slot
      max_w(ap >= a0 ? ap : a0, am, wi, wp);
      acc += g0 * (wi * wz);
      max_w(ap2, ap, wm, wz);  // y = x + o: (ap2 op ap) op a0, x the outer second slot
      max_w(ap2 >= ap ? ap2 : ap, a0, wi, wp);
      ca = acc + gp * wp;
    }
  } else if (op == G_ST2) {
    // y = st1(a) +- st2(b): each stencil's transpose of the cotangent.
    const T v1 = stencil_at(gout, c, nd.axis, st_transpose(nd.sk), kc<T>(nd.c0, nd.f0), g);
    const T v2 = stencil_at(gout, c, nd.axis2, st_transpose(nd.sk2), kc<T>(nd.h2, nd.fh2), g);
    ca = st_negates(nd.sk) ? -v1 : v1;
    cb = (st_negates(nd.sk2) != (nd.iop == G_SUB)) ? -v2 : v2;
  } else {   // G_SHIFT
    ca = gout[nbr(c, nd.axis, -nd.sk, g)];
  }
}

// A pointwise op's cotangents of a and b from y = its value and gg = y's
// cotangent (before the folded sum's sign and the epilogue's factor, which
// the kernel applies; exp reads ps exp(a) = y - pt itself).
template <typename T>
__device__ __forceinline__ void pw_grad(int op, const GNode& nd, T a, T b, T y, T gg, T& ca,
                                        T& cb) {
  ca = 0;
  cb = 0;
  switch (op) {
    case G_ADD: ca = gg; cb = gg; break;
    case G_SUB: ca = gg; cb = -gg; break;
    case G_MUL: ca = gg * b; cb = gg * a; break;
    case G_DIV:
      ca = gg / b;
      cb = -gg * a / (b * b);
      break;
    case G_MAX:
      ca = a > b ? gg : (a == b ? gg / (T)2 : (T)0);
      cb = b > a ? gg : (a == b ? gg / (T)2 : (T)0);
      break;
    case G_EXP: ca = gg * (y - kc<T>(nd.pt, nd.fpt)); break;   // ps exp(a) = y - pt
    case G_LOG: ca = gg / a; break;
    case G_LOG1P: ca = gg / ((T)1 + a); break;
    case G_SQRT: ca = gg / ((T)2 * y); break;
    case G_ABS: ca = a > (T)0 ? gg : (a < (T)0 ? -gg : (T)0); break;
    case G_AXPB: ca = kc<T>(nd.c0, nd.f0) * gg; break;
    case G_CLAMPMIN: ca = a >= kc<T>(nd.c0, nd.f0) ? gg : (T)0; break;
    case G_CLAMPMAX: ca = a <= kc<T>(nd.c0, nd.f0) ? gg : (T)0; break;
    default: break;
  }
}

// Pointwise transpose over n cells (the layout of g_forward_pw): the
// cotangents, scaled by the folded sum's sign and the epilogue's factor, are
// written (first contribution) or added into gA, gB, gC; a and b may be the
// same node (a's contribution first).
template <typename T, int OP>
__device__ __forceinline__ void pw_back_cell(const GNode& nd, T a, T b, T y, T gg, T sv, T sc,
                                             T& ca, T& cb, T& cc) {
  pw_grad(OP, nd, a, b, y, gg, ca, cb);
  if ((nd.ep && OP != G_EXP) || nd.pop == 3) {
    ca *= sv;
    cb *= sv;
  }
  cc = sc * gg;
}

template <typename T, int OP>
__global__ void g_backward_pw(GNode nd, const T* A, const T* B, const T* out, const T* gout,
                              T* gA, T* gB, T* gC, int wA, int wB, int wC, long long n, int vec) {
  const bool same = gA != nullptr && gA == gB;
  const T sv = kc<T>(nd.ps, nd.fps) * (nd.pop == 3 ? (T)-1 : (T)1);
  const T sc = kc<T>(nd.ps, nd.fps) * (nd.pop == 2 ? (T)-1 : (T)1);
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  auto put = [](int w, T v, T old) { return w ? v : old + v; };   // first write, or add
  if (vec) {
    for (; t < n / 4; t += stride) {
      const long long i = 4 * t;
      T a[4] = {0, 0, 0, 0}, b[4] = {0, 0, 0, 0}, y[4], gg[4], ca[4], cb[4], cc[4];
      T oa[4] = {0, 0, 0, 0}, ob[4] = {0, 0, 0, 0}, oc[4] = {0, 0, 0, 0};
      if (A) ld4(A, i, a);
      if (B) ld4(B, i, b);
      ld4(out, i, y);
      ld4(gout, i, gg);
      if (gA && !wA) ld4((const T*)gA, i, oa);
      if (gB && !wB && !same) ld4((const T*)gB, i, ob);
      if (gC && !wC) ld4((const T*)gC, i, oc);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        pw_back_cell<T, OP>(nd, a[k], b[k], y[k], gg[k], sv, sc, ca[k], cb[k], cc[k]);
        if (same) {
          oa[k] = put(wB, cb[k], put(wA, ca[k], oa[k]));
        } else {
          oa[k] = put(wA, ca[k], oa[k]);
          ob[k] = put(wB, cb[k], ob[k]);
        }
        oc[k] = put(wC, cc[k], oc[k]);
      }
      if (gA) st4(gA, i, oa);
      if (gB && !same) st4(gB, i, ob);
      if (gC) st4(gC, i, oc);
    }
  } else {
    for (; t < n; t += stride) {
      T ca, cb, cc;
      pw_back_cell<T, OP>(nd, A ? A[t] : (T)0, B ? B[t] : (T)0, out[t], gout[t], sv, sc, ca, cb,
                          cc);
      if (same) {
        gA[t] = put(wB, cb, put(wA, ca, wA ? (T)0 : gA[t]));
      } else {
        if (gA) gA[t] = put(wA, ca, wA ? (T)0 : gA[t]);
        if (gB) gB[t] = put(wB, cb, wB ? (T)0 : gB[t]);
      }
      if (gC) gC[t] = put(wC, cc, wC ? (T)0 : gC[t]);
    }
  }
}

// The first contribution a gradient receives in the reverse sweep writes it
// (wA, wB); later ones accumulate.  a and b may be the same node: a's
// contribution is applied first, as two sequential updates would.
template <typename T, int OP>
__global__ void g_backward(GNode nd, const T* A, const T* B, const T* out, const T* gout,
                           T* gA, T* gB, T* gC, int wA, int wB, int wC, Geo g) {
  GCell c0;
  if (!gcell(c0, g)) return;
  const bool same = gA != nullptr && gA == gB;
  // The factors of the epilogue and the folded sum: every transpose is linear
  // in gout, and C's cotangent is +-ps gout at the cell (C is neither a nor b).
  const T sv = kc<T>(nd.ps, nd.fps) * (nd.pop == 3 ? (T)-1 : (T)1);
  const T sc = kc<T>(nd.ps, nd.fps) * (nd.pop == 2 ? (T)-1 : (T)1);
  T ca[GZU], cb[GZU], oa[GZU], ob[GZU];
#pragma unroll
  for (int u = 0; u < GZU; ++u) {
    const GCell c = gcell_at(c0, u, g);
    if (c.k < g.nz) {
      bwd_value(OP, nd, A, B, out, gout, c, g, ca[u], cb[u]);
      // exp's transposes take the epilogue's factor from their own value.
      if ((nd.ep && OP != G_EXP && OP != G_STEXP) || nd.pop == 3) {
        ca[u] *= sv;
        cb[u] *= sv;
      }
      oa[u] = (gA && !wA) ? gA[c.idx] : (T)0;
      ob[u] = (gB && !wB && !same) ? gB[c.idx] : (T)0;
      if (gC) {
        const T v = sc * gout[c.idx];
        gC[c.idx] = wC ? v : gC[c.idx] + v;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < GZU; ++u) {
    const GCell c = gcell_at(c0, u, g);
    if (c.k < g.nz) {
      if (same) {
        T v = wA ? ca[u] : oa[u] + ca[u];
        gA[c.idx] = wB ? cb[u] : v + cb[u];
      } else {
        if (gA) gA[c.idx] = wA ? ca[u] : oa[u] + ca[u];
        if (gB) gB[c.idx] = wB ? cb[u] : ob[u] + cb[u];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// The same stencil-type kernels with four consecutive x-cells a thread (nx a
// multiple of 4, every array 16-byte aligned): each tap is one 16-byte load,
// the x taps come from the aligned 4-cell chunks left of, at and right of the
// thread's cells, and the per-thread index work is shared by four cells (the
// one-cell kernels are bound by their instruction issue).  Every lane takes
// the one-cell arithmetic, so the values are the same bit for bit.  SHIFT and
// NB3 here take offsets of one cell.
// ---------------------------------------------------------------------------
struct GCell4 {
  int i0, j, k;   // i0: the first of the four x-cells
  long long idx;  // index of cell i0
};

__device__ __forceinline__ bool gcell4(GCell4& c, const Geo& g) {
  c.i0 = 4 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
  c.j = blockIdx.y * blockDim.y + threadIdx.y;
  c.k = blockIdx.z * blockDim.z + threadIdx.z;
  if (c.i0 >= g.nx || c.j >= g.ny || c.k >= g.nz) return false;
  c.idx = (long long)c.k * g.sz + (long long)c.j * g.sy + c.i0;
  return true;
}

// t[o + K][l]: f at cell (i0 + l, j, k) + o e_axis, o = -K .. K (K <= 3).
template <int K, typename T>
__device__ __forceinline__ void tapsx4(const T* f, const GCell4& c, int axis, const Geo& g,
                                       T t[2 * K + 1][4]) {
  if (axis == 0) {
    const long long row = c.idx - c.i0;
    T L[4], M[4], R[4];
    ld4(f, row + wrap(c.i0 - 4, g.nx), L);
    ld4(f, c.idx, M);
    ld4(f, row + wrap(c.i0 + 4, g.nx), R);
#pragma unroll
    for (int o = -K; o <= K; ++o)
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int q = 4 + l + o;   // in the 12-cell window i0 - 4 .. i0 + 7
        t[o + K][l] = q < 4 ? L[q] : q < 8 ? M[q - 4] : R[q - 8];
      }
  } else {
    const long long st = axis == 1 ? g.sy : g.sz;
    const int pos = axis == 1 ? c.j : c.k, n = axis == 1 ? g.ny : g.nz;
    const bool inner = pos >= K && pos + K < n;
#pragma unroll
    for (int o = -K; o <= K; ++o)
      ld4(f, c.idx + (inner ? o * st : (long long)(wrap(pos + o, n) - pos) * st), t[o + K]);
  }
}
template <typename T>
__device__ __forceinline__ void taps7x4(const T* f, const GCell4& c, int axis, const Geo& g,
                                        T t[7][4]) {
  tapsx4<3>(f, c, axis, g, t);
}

// v[l]: f at cell (i0 + l, j, k) + o e_axis, one offset o in -1 .. 1.
template <typename T>
__device__ __forceinline__ void tap1x4(const T* f, const GCell4& c, int axis, int o,
                                       const Geo& g, T (&v)[4]) {
  if (axis == 0) {
    T t[3][4];
    tapsx4<1>(f, c, 0, g, t);
#pragma unroll
    for (int l = 0; l < 4; ++l) v[l] = o < 0 ? t[0][l] : o > 0 ? t[2][l] : t[1][l];
  } else {
    const long long st = axis == 1 ? g.sy : g.sz;
    const int pos = axis == 1 ? c.j : c.k, n = axis == 1 ? g.ny : g.nz;
    ld4(f, c.idx + (long long)(wrap(pos + o, n) - pos) * st, v);
  }
}

// Lane l's seven taps as one array.
template <typename T>
__device__ __forceinline__ void lane7(const T t[7][4], int l, T u[7]) {
#pragma unroll
  for (int o = 0; o < 7; ++o) u[o] = t[o][l];
}
// The tap at offset s = +-1 (or +-2 with d2) of lane l.
template <typename T>
__device__ __forceinline__ T tap1(const T t[7][4], int s, int l) {
  return s > 0 ? t[4][l] : t[2][l];
}
template <typename T>
__device__ __forceinline__ T tap2(const T t[7][4], int s, int l) {
  return s > 0 ? t[5][l] : t[1][l];
}

// FP32: at most 64 registers (4 blocks per SM): the transposes that gather
// two or three tap arrays spill about 100 bytes then, yet run faster than at
// 76-84 registers and 3 blocks (STBIN of a product 38 -> 21 us, STEXP 23 -> 16
// us at 128^3); the forward kernels taken with four cells stay under 64
// anyway.  FP64 (twice the registers a value) keeps the compiler's choice.
template <typename T, int OP>
__global__ void __launch_bounds__(GBX * GBY * GBZ, sizeof(T) == 4 ? 4 : 1)
    g_forward4(GNode nd, const T* A, const T* B, const T* C, T* out, const T* mesh, Geo g) {
  GCell4 c;
  if (!gcell4(c, g)) return;
  const T h = kc<T>(nd.c0, nd.f0);
  T r[4];
  if (OP == G_ZFIELD) {
    const T z = mesh[(long long)nd.sk * g.nz + c.k];
#pragma unroll
    for (int l = 0; l < 4; ++l) r[l] = z;
  } else if (OP == G_STMUL) {
    // The product formed as B's taps arrive: one tap array live.
    T ta[7][4];
    taps7x4(A, c, nd.axis, g, ta);
    {
      T tb[7][4];
      taps7x4(B, c, nd.axis, g, tb);
#pragma unroll
      for (int o = 0; o < 7; ++o)
#pragma unroll
        for (int l = 0; l < 4; ++l) ta[o][l] = ta[o][l] * tb[o][l];
    }
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      T u[7];
      lane7(ta, l, u);
      r[l] = st_comb(nd.sk, h, u);
    }
  } else if (OP == G_ST2) {
    // The two stencils one after the other: one tap array live.
    T s1[4];
    {
      T ta[7][4];
      taps7x4(A, c, nd.axis, g, ta);
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        T u[7];
        lane7(ta, l, u);
        s1[l] = st_comb(nd.sk, h, u);
      }
    }
    T tb[7][4];
    taps7x4(B, c, nd.axis2, g, tb);
    const T h2 = kc<T>(nd.h2, nd.fh2);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      T v[7];
      lane7(tb, l, v);
      const T s2 = st_comb(nd.sk2, h2, v);
      r[l] = nd.iop == G_ADD ? s1[l] + s2 : s1[l] - s2;
    }
  } else {
    T t[7][4];
    taps7x4(A, c, nd.axis, g, t);
    T b[4] = {0, 0, 0, 0};
    if (OP == G_STBIN) ld4(B, c.idx, b);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      if (OP == G_SHIFT) {
        r[l] = tap1(t, nd.sk, l);
      } else if (OP == G_NB3) {
        const T m = tap1(t, nd.sk, l), z = t[3][l], p = tap1(t, -nd.sk, l);
        if (nd.iop == G_ADD) {
          r[l] = (m + z) + p;
        } else {
          const T in = m >= z ? m : z;
          r[l] = in >= p ? in : p;
        }
      } else {
        T u[7];
        lane7(t, l, u);
        const T st = st_comb(nd.sk, h, u);
        r[l] = OP == G_STEXP ? exp(st) : OP == G_STBIN ? stbin_val(nd, st, b[l]) : st;
      }
    }
  }
  T cv[4] = {0, 0, 0, 0};
  if (nd.pop) ld4(C, c.idx, cv);
#pragma unroll
  for (int l = 0; l < 4; ++l) r[l] = finish(nd, r[l], cv[l]);
  st4(out, c.idx, r);
}

template <typename T, int OP>
__global__ void __launch_bounds__(GBX * GBY * GBZ, sizeof(T) == 4 ? 4 : 1)
    g_backward4(GNode nd, const T* A, const T* B, const T* out, const T* gout, T* gA, T* gB,
                T* gC, int wA, int wB, int wC, Geo g) {
  GCell4 c;
  if (!gcell4(c, g)) return;
  const T h = kc<T>(nd.c0, nd.f0);
  const int tk = st_transpose(nd.sk);
  const bool ng = st_negates(nd.sk);
  T ca[4] = {0, 0, 0, 0}, cb[4] = {0, 0, 0, 0}, gg[4];
  ld4(gout, c.idx, gg);
  if (OP == G_ST2) {
    T t1[7][4], t2[7][4];
    taps7x4(gout, c, nd.axis, g, t1);
    taps7x4(gout, c, nd.axis2, g, t2);
    const T h2 = kc<T>(nd.h2, nd.fh2);
    const bool n2 = st_negates(nd.sk2) != (nd.iop == G_SUB);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      T u[7], v[7];
      lane7(t1, l, u);
      lane7(t2, l, v);
      const T v1 = st_comb(tk, h, u), v2 = st_comb(st_transpose(nd.sk2), h2, v);
      ca[l] = ng ? -v1 : v1;
      cb[l] = n2 ? -v2 : v2;
    }
  } else if (OP == G_NB3) {
    T tg[7][4], ta[7][4];
    taps7x4(gout, c, nd.axis, g, tg);
    if (nd.iop != G_ADD) taps7x4(A, c, nd.axis, g, ta);
    const int o = nd.sk;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const T gm = tap1(tg, -o, l), g0 = tg[3][l], gp = tap1(tg, o, l);
      if (nd.iop == G_ADD) {
        ca[l] = (gm + g0) + gp;
      } else {
        const T a0 = ta[3][l], am = tap1(ta, -o, l), am2 = tap2(ta, -o, l);
        const T ap = tap1(ta, o, l), ap2 = tap2(ta, o, l);
        T wm, wz, wi, wp;
        max_w(a0, am, wm, wz);
        max_w(a0 >= am ? a0 : am, am2, wi, wp);
        T acc = gm * (wi * wm);
        max_w(ap, a0, wm, wz);
        max_w(ap >= a0 ? ap : a0, am, wi, wp);
        acc += g0 * (wi * wz);
        max_w(ap2, ap, wm, wz);
        max_w(ap2 >= ap ? ap2 : ap, a0, wi, wp);
        ca[l] = acc + gp * wp;
      }
    }
  } else if (OP == G_SHIFT) {
    T tg[7][4];
    taps7x4(gout, c, nd.axis, g, tg);
#pragma unroll
    for (int l = 0; l < 4; ++l) ca[l] = tap1(tg, -nd.sk, l);
  } else {
    // STENCIL, STBIN, STMUL, STEXP: the transposed stencil of gout, or of
    // gout times B (STBIN with a product) or times y - pt (STEXP).
    // One tap array live at a time (the product formed as its factor
    // arrives), then, for STBIN of a product, the stencil of A for cb.
    const bool prod = (OP == G_STBIN && nd.iop == G_MUL) || OP == G_STEXP;
    {
      T tg[7][4];
      taps7x4(gout, c, nd.axis, g, tg);
      if (prod) {
        T tb[7][4];
        taps7x4(OP == G_STEXP ? out : B, c, nd.axis, g, tb);
        const T pt = kc<T>(nd.pt, nd.fpt);
#pragma unroll
        for (int q = 0; q < 7; ++q)
#pragma unroll
          for (int l = 0; l < 4; ++l)
            tg[q][l] = OP == G_STEXP ? tg[q][l] * (tb[q][l] - pt) : tg[q][l] * tb[q][l];
      }
      T a[4] = {0, 0, 0, 0}, b[4] = {0, 0, 0, 0};
      if (OP == G_STMUL) {
        ld4(A, c.idx, a);
        ld4(B, c.idx, b);
      }
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        T u[7];
        lane7(tg, l, u);
        T v = st_comb(tk, h, u);
        if (ng) v = -v;
        if (OP == G_STBIN) {
          if (nd.iop == G_MUL) {
            ca[l] = v;
          } else {
            ca[l] = (nd.iop == G_SUB && nd.side) ? -v : v;
            cb[l] = (nd.iop == G_SUB && !nd.side) ? -gg[l] : gg[l];
          }
        } else if (OP == G_STMUL) {
          ca[l] = v * b[l];
          cb[l] = v * a[l];
        } else {
          ca[l] = v;
        }
      }
    }
    if (OP == G_STBIN && nd.iop == G_MUL) {
      T ta[7][4];
      taps7x4(A, c, nd.axis, g, ta);
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        T w[7];
        lane7(ta, l, w);
        cb[l] = gg[l] * st_comb(nd.sk, h, w);
      }
    }
  }
  const bool same = gA != nullptr && gA == gB;
  const T sv = kc<T>(nd.ps, nd.fps) * (nd.pop == 3 ? (T)-1 : (T)1);
  const T sc = kc<T>(nd.ps, nd.fps) * (nd.pop == 2 ? (T)-1 : (T)1);
  if ((nd.ep && OP != G_STEXP) || nd.pop == 3) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      ca[l] *= sv;
      cb[l] *= sv;
    }
  }
  auto put = [](int w, T v, T old) { return w ? v : old + v; };   // first write, or add
  T oa[4] = {0, 0, 0, 0}, ob[4] = {0, 0, 0, 0}, oc[4] = {0, 0, 0, 0};
  if (gA && !wA) ld4((const T*)gA, c.idx, oa);
  if (gB && !wB && !same) ld4((const T*)gB, c.idx, ob);
  if (gC && !wC) ld4((const T*)gC, c.idx, oc);
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    if (same) {
      oa[l] = put(wB, cb[l], put(wA, ca[l], oa[l]));
    } else {
      oa[l] = put(wA, ca[l], oa[l]);
      ob[l] = put(wB, cb[l], ob[l]);
    }
    oc[l] = put(wC, sc * gg[l], oc[l]);
  }
  if (gA) st4(gA, c.idx, oa);
  if (gB && !same) st4(gB, c.idx, ob);
  if (gC) st4(gC, c.idx, oc);
}

// The quench's kernels with four x-cells a thread (the same per-lane
// arithmetic as g_quench_f, g_quench_q, g_quench_b1 and g_quench_b3).
template <typename T>
__global__ void g_quench_f4(GNode nd, const T* A, T* out, Geo g) {
  GCell4 c;
  if (!gcell4(c, g)) return;
  const T iq = (T)1 / kc<T>(nd.c0, nd.f0), qlim = kc<T>(nd.c1, nd.f1);
  const T eps = kc<T>(nd.c2, nd.f2);
  T ta[2][5][4];   // T at offsets -2 .. 2 along each axis slot
  tapsx4<2>(A, c, nd.axis, g, ta[0]);
  if (nd.sk >= 0) tapsx4<2>(A, c, nd.sk, g, ta[1]);
  T r[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const T fac = quench_fac<T>(
        [&](int t, int, int s) {
          return q_val(ta[t][s + 1][l], ta[t][s + 2][l], ta[t][s + 3][l], iq, eps, (T*)nullptr);
        },
        nd.axis, nd.sk, (T*)nullptr);
    r[l] = ta[0][2][l] * (fac > qlim ? qlim : fac);
  }
  st4(out, c.idx, r);
}

template <typename T>
__global__ void g_quench_q4(GNode nd, const T* A, T* Q, Geo g) {
  GCell4 c;
  if (!gcell4(c, g)) return;
  const T iq = (T)1 / kc<T>(nd.c0, nd.f0), eps = kc<T>(nd.c2, nd.f2);
  for (int t = 0; t < 2; ++t) {
    const int ax = t == 0 ? nd.axis : nd.sk;
    if (ax < 0) continue;
    T ta[3][4];
    tapsx4<1>(A, c, ax, g, ta);
    T q[4], d0[4], d1[4], d2[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      T dq[3];
      q[l] = q_val(ta[0][l], ta[1][l], ta[2][l], iq, eps, dq);
      d0[l] = dq[0];
      d1[l] = dq[1];
      d2[l] = dq[2];
    }
    st4(Q + (long long)(4 * t) * g.n, c.idx, q);
    st4(Q + (long long)(4 * t + 1) * g.n, c.idx, d0);
    st4(Q + (long long)(4 * t + 2) * g.n, c.idx, d1);
    st4(Q + (long long)(4 * t + 3) * g.n, c.idx, d2);
  }
}

template <typename T>
__global__ void g_quench_b1_4(GNode nd, const T* A, const T* Q, const T* gout, T* S, Geo g) {
  GCell4 c;
  if (!gcell4(c, g)) return;
  const T qlim = kc<T>(nd.c1, nd.f1);
  T tq[2][3][4];   // q at offsets -1 .. 1 along each axis slot
  tapsx4<1>(Q, c, nd.axis, g, tq[0]);
  if (nd.sk >= 0) tapsx4<1>(Q + 4 * g.n, c, nd.sk, g, tq[1]);
  T a[4], gg[4];
  ld4(A, c.idx, a);
  ld4(gout, c.idx, gg);
  T s0[4], sw[6][4];
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    T wq[6];
    const T fac = quench_fac<T>([&](int t, int, int s) { return tq[t][s + 1][l]; }, nd.axis,
                                nd.sk, wq);
    const T C = fac > qlim ? qlim : fac;
    const T dC = fac <= qlim ? (T)1 : (T)0;
    const T base = gg[l] * a[l] * dC;
    s0[l] = gg[l] * C;
#pragma unroll
    for (int j = 0; j < 6; ++j) sw[j][l] = base * wq[j];
  }
  st4(S, c.idx, s0);
#pragma unroll
  for (int j = 0; j < 6; ++j) st4(S + (long long)(1 + j) * g.n, c.idx, sw[j]);
}

template <typename T>
__global__ void g_quench_b3_4(GNode nd, const T* Q, const T* S, T* gA, int wA, Geo g) {
  GCell4 c;
  if (!gcell4(c, g)) return;
  T acc[4];
  ld4(S, c.idx, acc);
  for (int t = 0; t < 2; ++t) {
    const int ax = t == 0 ? nd.axis : nd.sk;
    if (ax < 0) continue;
    T ts[3][5][4];   // S of q position p = -1 .. 1 at offsets -2 .. 2
#pragma unroll
    for (int p = 0; p < 3; ++p) tapsx4<2>(S + (long long)(1 + 3 * t + p) * g.n, c, ax, g, ts[p]);
    T td[3][4];   // d q(z) / d T at its tap 1 - r, z at offsets r = -1 .. 1
#pragma unroll
    for (int r = -1; r <= 1; ++r)
      tap1x4(Q + (long long)(4 * t + 2 - r) * g.n, c, ax, r, g, td[r + 1]);
#pragma unroll
    for (int r = -1; r <= 1; ++r)
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        T qbar = 0;
#pragma unroll
        for (int p = -1; p <= 1; ++p) qbar += ts[p + 1][r - p + 2][l];
        acc[l] += qbar * td[r + 1][l];
      }
  }
  if (!wA) {
    T o[4];
    ld4((const T*)gA, c.idx, o);
#pragma unroll
    for (int l = 0; l < 4; ++l) acc[l] = o[l] + acc[l];
  }
  st4(gA, c.idx, acc);
}

// Horizontal-plane mean (G_PMEAN): one block per z sums its plane in a fixed
// order; the broadcast writes (or, for the transpose, adds) sum / (nx ny).
// The mean is linear and symmetric, so its transpose is the same mean.
template <typename T>
__global__ void g_plane_sum(const T* A, T* psum, Geo g) {
  __shared__ T sm[256];
  const int kz = blockIdx.x;
  const long long m = (long long)g.nx * g.ny;
  T acc = 0;
  for (long long i = threadIdx.x; i < m; i += blockDim.x) acc += A[(long long)kz * g.sz + i];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) psum[kz] = sm[0];
}

template <typename T>
__global__ void g_plane_bcast(const T* psum, T* out, int add, Geo g) {
  GCell c0;
  if (!gcell(c0, g)) return;
  for (int u = 0; u < GZU; ++u) {
    const GCell c = gcell_at(c0, u, g);
    if (c.k >= g.nz) break;
    const T v = psum[c.k] / (T)((double)g.nx * g.ny);
    out[c.idx] = add ? out[c.idx] + v : v;
  }
}

// dst[k] += src[k] for up to eight arrays in one launch (blockIdx.y = k).
template <typename T>
struct Add8 {
  T* dst[8];
  const T* src[8];
};
template <typename T>
__global__ void g_add_into8(Add8<T> p, long long n, int vec) {
  T* dst = p.dst[blockIdx.y];
  const T* src = p.src[blockIdx.y];
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (vec) {   // four elements a thread through 16-byte accesses
    for (; t < n / 4; t += stride) {
      T a[4], b[4];
      ld4((const T*)dst, 4 * t, a);
      ld4(src, 4 * t, b);
#pragma unroll
      for (int l = 0; l < 4; ++l) a[l] += b[l];
      st4(dst, 4 * t, a);
    }
  } else {
    for (; t < n; t += stride) dst[t] += src[t];
  }
}

}  // namespace stg
