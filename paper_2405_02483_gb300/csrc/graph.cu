// Op-graph engine (see graph.cuh): forward and transpose kernels of every
// primitive, the right-hand-side graph of the MHD equations, and the executor.
#include <math.h>

#include <algorithm>

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

// Periodic neighbour of cell c along an axis (shifted by o).
__device__ __forceinline__ long long nbr(const GCell& c, int axis, int o, const Geo& g) {
  if (axis == 0) return c.idx + (wrap(c.i + o, g.nx) - c.i);
  if (axis == 1) return c.idx + (long long)(wrap(c.j + o, g.ny) - c.j) * g.sy;
  return c.idx + (long long)(wrap(c.k + o, g.nz) - c.k) * g.sz;
}

// Stencil value at c: up/dn are eq. (interp) to i+1/2 and i-1/2; ddup/dddn
// are eq. (deriv) to i+1/2 and i-1/2, divided by the spacing h.
template <typename T>
__device__ __forceinline__ T stencil_at(const T* f, const GCell& c, int axis, int kind, T h,
                                        const Geo& g) {
  const T IA = (T)STG_IA, IB = (T)STG_IB, IC = (T)STG_IC;
  const T DA = (T)STG_DA, DB = (T)STG_DB, DC = (T)STG_DC;
  T m3 = f[nbr(c, axis, -3, g)], m2 = f[nbr(c, axis, -2, g)], m1 = f[nbr(c, axis, -1, g)];
  T z0 = f[c.idx], p1 = f[nbr(c, axis, 1, g)], p2 = f[nbr(c, axis, 2, g)],
    p3 = f[nbr(c, axis, 3, g)];
  switch (kind) {
    case ST_UP: return IA * (z0 + p1) + IB * (m1 + p2) + IC * (m2 + p3);
    case ST_DN: return IA * (m1 + z0) + IB * (m2 + p1) + IC * (m3 + p2);
    case ST_DDUP: return (DA * (p1 - z0) + DB * (p2 - m1) + DC * (p3 - m2)) / h;
    default: return (DA * (z0 - m1) + DB * (p1 - m2) + DC * (p2 - m3)) / h;
  }
}

// The same stencil of the values v(idx) of a functor at the taps.
template <typename T, class V>
__device__ __forceinline__ T stencil_fn(V v, const GCell& c, int axis, int kind, T h,
                                        const Geo& g) {
  const T IA = (T)STG_IA, IB = (T)STG_IB, IC = (T)STG_IC;
  const T DA = (T)STG_DA, DB = (T)STG_DB, DC = (T)STG_DC;
  T m3 = v(nbr(c, axis, -3, g)), m2 = v(nbr(c, axis, -2, g)), m1 = v(nbr(c, axis, -1, g));
  T z0 = v(c.idx), p1 = v(nbr(c, axis, 1, g)), p2 = v(nbr(c, axis, 2, g)),
    p3 = v(nbr(c, axis, 3, g));
  switch (kind) {
    case ST_UP: return IA * (z0 + p1) + IB * (m1 + p2) + IC * (m2 + p3);
    case ST_DN: return IA * (m1 + z0) + IB * (m2 + p1) + IC * (m3 + p2);
    case ST_DDUP: return (DA * (p1 - z0) + DB * (p2 - m1) + DC * (p3 - m2)) / h;
    default: return (DA * (z0 - m1) + DB * (p1 - m2) + DC * (p2 - m3)) / h;
  }
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
// M = |T| + eps max3 |T| (eps = c2 >= 0), or M = max3 |T| (c2 < 0).  Its transpose follows the rules of the primitive nodes it
// stands for: a max splits the gradient evenly on a tie (pairwise, the inner
// pair first), |x|' = sign x with sign 0 = 0, the clamp passes the gradient
// where fac <= qlim.
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

// q at z = c + s e_ax, and (dq) its derivatives with respect to T at z-1, z,
// z+1 (through D2 T and through M).
template <typename T>
__device__ __forceinline__ T q_at(const T* A, const GCell& c, int ax, int s, T iq, T eps,
                                  const Geo& g, T* dq) {
  const T vm = A[nbr(c, ax, s - 1, g)], v0 = A[nbr(c, ax, s, g)], vp = A[nbr(c, ax, s + 1, g)];
  const T d2 = (vp - (T)2 * v0) + vm, a2 = fabs(d2);
  const T am = fabs(vm), a0 = fabs(v0), ap = fabs(vp);
  const T inner = am >= a0 ? am : a0;
  const T M3 = inner >= ap ? inner : ap;
  // M = cM max3|T| + cP |T|.
  const T cM = eps < (T)0 ? (T)1 : eps, cP = eps < (T)0 ? (T)0 : (T)1;
  const T M = eps < (T)0 ? M3 : a0 + eps * M3;
  const T den = (M + a2 * iq) + (T)1e-30;
  const T q = a2 / den;
  if (dq) {
    T wim, wi0, woi, wop;
    max_w(am, a0, wim, wi0);
    max_w(inner, ap, woi, wop);
    const T dq_da2 = (T)1 / den + iq * (-a2 / (den * den));
    const T dq_dM = -a2 / (den * den);
    const T sd = sgn(d2);
    dq[0] = dq_da2 * sd + dq_dM * (cM * (woi * wim)) * sgn(vm);
    dq[1] = dq_da2 * sd * (T)-2 + dq_dM * (cM * (woi * wi0) + cP) * sgn(v0);
    dq[2] = dq_da2 * sd + dq_dM * (cM * wop) * sgn(vp);
  }
  return q;
}

// fac at c, and (when wq) the weights of the three q of each axis in fac:
// wq[3 t + p + 1] for axis t and position p.
template <typename T>
__device__ __forceinline__ T quench_fac(const T* A, const GCell& c, int a0, int a1, T iq, T eps,
                                        const Geo& g, T* wq) {
  T m[2] = {0, 0}, w[2][3];
  for (int t = 0; t < 2; ++t) {
    const int ax = t == 0 ? a0 : a1;
    if (ax < 0) continue;
    const T qm = q_at(A, c, ax, -1, iq, eps, g, (T*)nullptr),
            q0 = q_at(A, c, ax, 0, iq, eps, g, (T*)nullptr),
            qp = q_at(A, c, ax, 1, iq, eps, g, (T*)nullptr);
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

// Transpose, first pass (per output cell y): S0 = gbar C (the product's own
// term) and S[1 + 3 t + p + 1] = gbar T dC/dfac dfac/dq, the cotangent each
// q of axis t at position p receives from y.
template <typename T>
__global__ void g_quench_b1(GNode nd, const T* A, const T* gout, T* S, Geo g) {
  GCell c0;
  if (!gcell(c0, g)) return;
  const T iq = (T)1 / (T)nd.c0, qlim = (T)nd.c1;
  for (int u = 0; u < GZU; ++u) {
    const GCell c = gcell_at(c0, u, g);
    if (c.k >= g.nz) break;
    T wq[6];
    const T fac = quench_fac(A, c, nd.axis, nd.sk, iq, (T)nd.c2, g, wq);
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
__global__ void g_quench_b3(GNode nd, const T* A, const T* S, T* gA, int wA, Geo g) {
  GCell c0;
  if (!gcell(c0, g)) return;
  const T iq = (T)1 / (T)nd.c0;
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
        T dq[3];
        q_at(A, c, ax, r, iq, (T)nd.c2, g, dq);
        acc += qbar * dq[1 - r];
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
    const T fac = quench_fac(A, c, nd.axis, nd.sk, (T)1 / (T)nd.c0, (T)nd.c2, g, (T*)nullptr);
    out[c.idx] = A[c.idx] * (fac > (T)nd.c1 ? (T)nd.c1 : fac);
  }
}

template <typename T>
__device__ __forceinline__ T fwd_value(int op, const GNode& nd, const T* A, const T* B,
                                       const T* mesh, const GCell& c, const Geo& g) {
  const long long idx = c.idx;
  switch (op) {
    case G_STENCIL: return stencil_at(A, c, nd.axis, nd.sk, (T)nd.c0, g);
    case G_STBIN: {
      const T st = stencil_at(A, c, nd.axis, nd.sk, (T)nd.c0, g), b = B[idx];
      if (nd.iop == G_MUL) return st * b;
      if (nd.iop == G_ADD) return nd.side ? b + st : st + b;
      return nd.side ? b - st : st - b;     // G_SUB
    }
    case G_STMUL:
      return stencil_fn<T>([&](long long j) { return A[j] * B[j]; }, c, nd.axis, nd.sk,
                           (T)nd.c0, g);
    case G_SHIFT: return A[nbr(c, nd.axis, nd.sk, g)];
    case G_ADD: return A[idx] + B[idx];
    case G_SUB: return A[idx] - B[idx];
    case G_MUL: return A[idx] * B[idx];
    case G_DIV: return A[idx] / B[idx];
    case G_MAX: return A[idx] >= B[idx] ? A[idx] : B[idx];
    case G_EXP: return exp(A[idx]);
    case G_LOG: return log(A[idx]);
    case G_LOG1P: return log1p(A[idx]);
    case G_SQRT: return sqrt(A[idx]);
    case G_ABS: return fabs(A[idx]);
    case G_AXPB: return (T)nd.c0 * A[idx] + (T)nd.c1;
    case G_CLAMPMIN: return A[idx] < (T)nd.c0 ? (T)nd.c0 : A[idx];
    case G_CLAMPMAX: return A[idx] > (T)nd.c0 ? (T)nd.c0 : A[idx];
    case G_STEP: return A[idx] > (T)nd.c0 ? (T)1 : (T)0;
    case G_ZFIELD: return mesh[(long long)nd.sk * g.nz + c.k];
    default: return (T)nd.c0;  // G_CONST
  }
}

// Every node but G_QUENCH (g_quench_f) and G_PMEAN; one instance per op.
template <typename T, int OP>
__global__ void g_forward(GNode nd, const T* A, const T* B, T* out, const T* mesh, Geo g) {
  GCell c0;
  if (!gcell(c0, g)) return;
  T r[GZU];
#pragma unroll
  for (int u = 0; u < GZU; ++u) {
    const GCell c = gcell_at(c0, u, g);
    if (c.k < g.nz) r[u] = fwd_value(OP, nd, A, B, mesh, c, g);
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
    T v = stencil_at(gout, c, nd.axis, st_transpose(kind), (T)nd.c0, g);
    ca = st_negates(kind) ? -v : v;
  } else if (op == G_STBIN) {
    // y = st(a) (op) b: the stencil's transpose of the cotangent of st(a),
    // which is g (add), -+g (sub) or g b (mul) at each tap.
    const int tk = st_transpose(nd.sk);
    const T sg = st_negates(nd.sk) ? (T)-1 : (T)1;
    const T gg = gout[idx];
    if (nd.iop == G_MUL) {
      ca = sg * stencil_fn<T>([&](long long j) { return gout[j] * B[j]; }, c, nd.axis, tk,
                              (T)nd.c0, g);
      cb = gg * stencil_at(A, c, nd.axis, nd.sk, (T)nd.c0, g);
    } else {
      const T v = sg * stencil_at(gout, c, nd.axis, tk, (T)nd.c0, g);
      const bool neg_st = nd.iop == G_SUB && nd.side;    // b - st
      const bool neg_b = nd.iop == G_SUB && !nd.side;    // st - b
      ca = neg_st ? -v : v;
      cb = neg_b ? -gg : gg;
    }
  } else if (op == G_STMUL) {
    // y = st(a b): the transposed stencil of g, times the other factor.
    T v = stencil_at(gout, c, nd.axis, st_transpose(nd.sk), (T)nd.c0, g);
    if (st_negates(nd.sk)) v = -v;
    ca = v * B[idx];
    cb = v * A[idx];
  } else if (op == G_SHIFT) {
    ca = gout[nbr(c, nd.axis, -nd.sk, g)];
  } else {
    const T gg = gout[idx];
    switch (op) {
      case G_ADD: ca = gg; cb = gg; break;
      case G_SUB: ca = gg; cb = -gg; break;
      case G_MUL: ca = gg * B[idx]; cb = gg * A[idx]; break;
      case G_DIV: {
        T a = A[idx], b = B[idx];
        ca = gg / b;
        cb = -gg * a / (b * b);
        break;
      }
      case G_MAX: {
        T a = A[idx], b = B[idx];
        ca = a > b ? gg : (a == b ? gg / (T)2 : (T)0);
        cb = b > a ? gg : (a == b ? gg / (T)2 : (T)0);
        break;
      }
      case G_EXP: ca = gg * out[idx]; break;
      case G_LOG: ca = gg / A[idx]; break;
      case G_LOG1P: ca = gg / ((T)1 + A[idx]); break;
      case G_SQRT: ca = gg / ((T)2 * out[idx]); break;
      case G_ABS: {
        T a = A[idx];
        ca = a > (T)0 ? gg : (a < (T)0 ? -gg : (T)0);
        break;
      }
      case G_AXPB: ca = (T)nd.c0 * gg; break;
      case G_CLAMPMIN: ca = A[idx] >= (T)nd.c0 ? gg : (T)0; break;
      case G_CLAMPMAX: ca = A[idx] <= (T)nd.c0 ? gg : (T)0; break;
      default: break;
    }
  }
}

// The first contribution a gradient receives in the reverse sweep writes it
// (wA, wB); later ones accumulate.  a and b may be the same node: a's
// contribution is applied first, as two sequential updates would.
template <typename T, int OP>
__global__ void g_backward(GNode nd, const T* A, const T* B, const T* out, const T* gout,
                           T* gA, T* gB, int wA, int wB, Geo g) {
  GCell c0;
  if (!gcell(c0, g)) return;
  const bool same = gA != nullptr && gA == gB;
  T ca[GZU], cb[GZU], oa[GZU], ob[GZU];
#pragma unroll
  for (int u = 0; u < GZU; ++u) {
    const GCell c = gcell_at(c0, u, g);
    if (c.k < g.nz) {
      bwd_value(OP, nd, A, B, out, gout, c, g, ca[u], cb[u]);
      oa[u] = (gA && !wA) ? gA[c.idx] : (T)0;
      ob[u] = (gB && !wB && !same) ? gB[c.idx] : (T)0;
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

template <typename T>
__global__ void g_add_into(T* dst, const T* src, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] += src[i];
}

// ---------------------------------------------------------------------------
// The right-hand side, eqs. (mass), (mom), (itv), (ien), (vdiss), (indu),
// (ohm), written on the stored deviations f' (full value ref + f').
// ---------------------------------------------------------------------------
// Every node is a whole-array pass whose launch, ramp and tail cost as much as
// its bytes, so a stencil that feeds one sum, difference or product, and a
// product that feeds one stencil, are merged into one node (G_STBIN, G_STMUL):
// the pair's intermediate array and launches go away, and the fused node's
// transpose is the pair's (the stencil's gather-form transpose of the
// cotangent, times the other factor where there is one).  A node used twice,
// or as an output, keeps its array.  The graph is then compacted.
static void fuse_stencil_pairs(GraphDef& G) {
  const int nn = (int)G.nodes.size();
  std::vector<int> uses(nn, 0);
  for (const GNode& nd : G.nodes) {
    if (nd.a >= 0) ++uses[nd.a];
    if (nd.b >= 0) ++uses[nd.b];
  }
  for (int k = 0; k < 8; ++k) uses[G.out[k]] += 2;   // outputs keep their arrays
  std::vector<char> dead(nn, 0);
  for (int i = 0; i < nn; ++i) {
    GNode& nd = G.nodes[i];
    if (nd.op == G_ADD || nd.op == G_SUB || nd.op == G_MUL) {
      for (int side = 0; side < 2; ++side) {
        const int src = side == 0 ? nd.a : nd.b;
        if (src < 0 || dead[src] || G.nodes[src].op != G_STENCIL || uses[src] != 1) continue;
        const GNode st = G.nodes[src];
        GNode f = nd;
        f.op = G_STBIN;
        f.iop = nd.op;
        f.side = side;
        f.a = st.a;
        f.b = side == 0 ? nd.b : nd.a;
        f.axis = st.axis;
        f.sk = st.sk;
        f.c0 = st.c0;
        f.c1 = 0;
        nd = f;
        dead[src] = 1;
        break;
      }
    } else if (nd.op == G_STENCIL && nd.a >= 0 && !dead[nd.a] && G.nodes[nd.a].op == G_MUL &&
               uses[nd.a] == 1) {
      const GNode m = G.nodes[nd.a];
      dead[nd.a] = 1;
      nd.op = G_STMUL;
      nd.a = m.a;
      nd.b = m.b;
    }
  }
  // Compact: drop the absorbed nodes and renumber every reference.
  std::vector<int> id(nn, -1);
  std::vector<GNode> kept;
  for (int i = 0; i < nn; ++i)
    if (!dead[i]) {
      id[i] = (int)kept.size();
      kept.push_back(G.nodes[i]);
    }
  for (GNode& nd : kept) {
    if (nd.a >= 0) nd.a = id[nd.a];
    if (nd.b >= 0) nd.b = id[nd.b];
  }
  for (int k = 0; k < 8; ++k) {
    G.in[k] = id[G.in[k]];
    G.out[k] = id[G.out[k]];
  }
  G.nodes.swap(kept);
  G.memo.clear();
}

void build_rhs_graph(GraphDef& G, const stagger_grid& gr, const stagger_params& p) {
  G.nodes.clear();
  G.memo.clear();
  const int X = 0, Y = 1, Z = 2;
  const double h[3] = {gr.dx, gr.dy, gr.dz};
  const int nn[3] = {gr.nx, gr.ny, gr.nz};
  // A stretched z (R19): the mesh's dl_min takes its smallest z cell; z
  // derivatives are index-space stencils times 1/dz at the output (centre
  // after ddup, face after dddn); lengths and dl_min are local there.
  const bool zs = p.zc != nullptr;
  double zcmin = 1e300, dlxy = 1e300;
  for (int k = 0; zs && k < gr.nz; ++k) zcmin = std::min(zcmin, p.zc[k]);
  double dlmin = 1e300, any = 0;
  for (int a = 0; a < 3; ++a)
    if (nn[a] > 1) {
      dlmin = std::min(dlmin, (a == 2 && zs) ? zcmin : h[a]);
      if (a < 2) dlxy = std::min(dlxy, h[a]);
      any = 1;
    }
  if (!any) dlmin = std::min(h[0], std::min(h[1], h[2]));
  double sp[3];
  for (int a = 0; a < 3; ++a) sp[a] = nn[a] > 1 ? h[a] : dlmin;
  G.mesh.clear();
  int JC = -1, JF = -1, HC = -1, HF = -1, DLC = -1;
  if (zs) {
    const int nz = gr.nz;
    G.mesh.resize((size_t)5 * nz);
    for (int k = 0; k < nz; ++k) {
      G.mesh[k] = 1.0 / p.zc[k];
      G.mesh[nz + k] = 1.0 / p.zf[k];
      G.mesh[2 * nz + k] = p.zc[k];
      G.mesh[3 * nz + k] = p.zf[k];
      G.mesh[4 * nz + k] = std::min(dlxy, p.zc[k]);
    }
    JC = G.zfield(0);
    JF = G.zfield(1);
    HC = G.zfield(2);
    HF = G.zfield(3);
    DLC = G.zfield(4);
  }
  auto ddup = [&](int a, int ax) {
    return (zs && ax == 2) ? G.mul(G.st(ST_DDUP, a, ax, 1.0), JC) : G.st(ST_DDUP, a, ax, h[ax]);
  };
  auto dddn = [&](int a, int ax) {
    return (zs && ax == 2) ? G.mul(G.st(ST_DDDN, a, ax, 1.0), JF) : G.st(ST_DDDN, a, ax, h[ax]);
  };
  // x * (local dl_min) and x * c * length: a constant on a uniform mesh.
  auto times_dl = [&](int a, double c) {
    return zs ? G.mul(G.axpb(a, c, 0.0), DLC) : G.axpb(a, c * dlmin, 0.0);
  };
  auto up = [&](int a, int ax) { return G.up(a, ax); };
  auto dn = [&](int a, int ax) { return G.dn(a, ax); };
  auto full = [&](int a, double ref) { return ref != 0.0 ? G.axpb(a, 1.0, ref) : a; };
  auto neg = [&](int a) { return G.axpb(a, -1.0, 0.0); };

  int fin[8];
  for (int k = 0; k < 8; ++k) fin[k] = G.input(k);
  const double r0 = p.ref[0], E0 = p.ref[4];
  int rd = fin[0], Ed = fin[4];
  int r = full(rd, r0), E = full(Ed, E0);
  int pf[3], B[3], Bd[3];
  for (int d = 0; d < 3; ++d) {
    pf[d] = full(fin[1 + d], p.ref[1 + d]);
    Bd[d] = fin[5 + d];
    B[d] = full(Bd[d], p.ref[5 + d]);
  }

  // Primitives; faces and edges by log interpolation of rho (do_loginterp).
  // lr = ln(rho / r0) keeps FP32 resolution of small density deviations.
  int lr = -1;
  auto dens = [&](int t) {  // density from an interpolated lr (or rho') value
    if (p.log_interp) return r0 > 0 ? G.axpb(G.ex(t), r0, 0.0) : G.ex(t);
    return full(t, r0);
  };
  if (p.log_interp) lr = r0 > 0 ? G.lg1p(G.axpb(rd, 1.0 / r0, 0.0)) : G.lg(r);
  int lsrc = p.log_interp ? lr : rd;
  int rf[3], u[3];
  for (int d = 0; d < 3; ++d) {
    rf[d] = dens(dn(lsrc, d));
    u[d] = G.div(pf[d], rf[d]);
  }
  const double gm1 = p.gamma - 1.0;
  int Pd = G.axpb(Ed, gm1, 0.0);
  int P = G.axpb(Ed, gm1, gm1 * E0);
  int e = G.div(E, r);
  // e - e0 with e0 = E0/r0: (E' - e0 r') / r, its derivatives equal those of e.
  int ed = r0 > 0 ? G.div(G.sub(Ed, G.axpb(rd, E0 / r0, 0.0)), r) : e;
  int divu = G.add(G.add(ddup(u[X], X), ddup(u[Y], Y)), ddup(u[Z], Z));

  // Current J = curl B on edges (mu = 1).
  int Jx = G.sub(dddn(Bd[Z], Y), dddn(Bd[Y], Z));
  int Jy = G.sub(dddn(Bd[X], Z), dddn(Bd[Z], X));
  int Jz = G.sub(dddn(Bd[Y], X), dddn(Bd[X], Y));

  // Ideal E = -u x B, eq. (ohm).
  int Ex = neg(G.sub(G.mul(dn(u[Y], Z), dn(B[Z], Y)), G.mul(dn(u[Z], Y), dn(B[Y], Z))));
  int Ey = neg(G.sub(G.mul(dn(u[Z], X), dn(B[X], Z)), G.mul(dn(u[X], Z), dn(B[Z], X))));
  int Ez = neg(G.sub(G.mul(dn(u[X], Y), dn(B[Y], X)), G.mul(dn(u[Y], X), dn(B[X], Y))));

  const bool visc = p.nu_const > 0 || p.nu1 > 0 || p.nu2 > 0 || p.nu3 > 0 || p.csmag > 0;
  int Q = -1, txx = -1, tyy = -1, tzz = -1, txy = -1, tyz = -1, tzx = -1;
  int ediff[3] = {-1, -1, -1};
  if (visc) {
    int nxx, nyy, nzz, nxy, nyz, nzx;
    if (p.nu_const > 0) {
      nxx = nyy = nzz = nxy = nyz = nzx = G.cnst(p.nu_const);
    } else {
      // eq. (RMnu): nu1 |u| + nu3 (c_s + c_A) + nu2 dl_min max(0, -div u).
      int ucx = up(u[X], X), ucy = up(u[Y], Y), ucz = up(u[Z], Z);
      int uc2 = G.add(G.add(G.mul(ucx, ucx), G.mul(ucy, ucy)), G.mul(ucz, ucz));
      int bcx = up(B[X], X), bcy = up(B[Y], Y), bcz = up(B[Z], Z);
      int B2 = G.add(G.add(G.mul(bcx, bcx), G.mul(bcy, bcy)), G.mul(bcz, bcz));
      int nu = -1;
      auto acc = [&](int t) { nu = nu < 0 ? t : G.add(nu, t); };
      if (p.nu1 > 0) acc(G.axpb(G.sq(uc2), p.nu1, 0.0));
      if (p.nu3 > 0) {
        int cs = G.sq(G.div(G.axpb(P, p.gamma, 0.0), r));
        int ca = G.sq(G.div(B2, r));
        acc(G.axpb(G.add(cs, ca), p.nu3, 0.0));
      }
      if (p.nu2 > 0) acc(times_dl(G.cmin(neg(divu), 0.0), p.nu2));
      if (p.csmag > 0) {
        // eq. (nusmag): dl_min Csmag [2 (S_ii^2 - (div u)^2/3 + S_ij^2, i != j)]^1/2.
        int sxx = ddup(u[X], X), syy = ddup(u[Y], Y), szz = ddup(u[Z], Z);
        int sxy = G.axpb(G.add(dddn(u[X], Y), dddn(u[Y], X)), 0.5, 0.0);
        int syz = G.axpb(G.add(dddn(u[Y], Z), dddn(u[Z], Y)), 0.5, 0.0);
        int szx = G.axpb(G.add(dddn(u[Z], X), dddn(u[X], Z)), 0.5, 0.0);
        int dia = G.add(G.add(G.mul(sxx, sxx), G.mul(syy, syy)), G.mul(szz, szz));
        dia = G.sub(dia, G.axpb(G.mul(divu, divu), 1.0 / 3.0, 0.0));
        int offd = G.add(G.add(up(up(G.mul(sxy, sxy), X), Y), up(up(G.mul(syz, syz), Y), Z)),
                         up(up(G.mul(szx, szx), Z), X));
        int s2 = G.add(dia, G.axpb(offd, 2.0, 0.0));
        acc(times_dl(G.sq(G.axpb(G.cmin(s2, 0.0), 2.0, 0.0)), p.csmag));
      }
      // <nu>_{max smooth}: 3-cell max along x, y, z, then 3-cell mean.
      for (int ax = 0; ax < 3; ++ax) nu = G.maxi(G.maxi(G.shift(nu, ax, -1), nu), G.shift(nu, ax, 1));
      for (int ax = 0; ax < 3; ++ax)
        nu = G.axpb(G.add(G.add(G.shift(nu, ax, -1), nu), G.shift(nu, ax, 1)), 1.0 / 3.0, 0.0);
      int lnu = G.lg(G.cmin(nu, 1e-30));
      nxx = G.axpb(nu, sp[X], 0.0);
      nyy = G.axpb(nu, sp[Y], 0.0);
      nxy = G.axpb(G.ex(dn(dn(lnu, X), Y)), std::max(sp[X], sp[Y]), 0.0);
      if (zs) {   // z length at the centre; the Ex, Ey edges sit on z faces
        nzz = G.mul(nu, HC);
        nyz = G.mul(G.ex(dn(dn(lnu, Y), Z)), G.maxi(G.cnst(sp[Y]), HF));
        nzx = G.mul(G.ex(dn(dn(lnu, Z), X)), G.maxi(HF, G.cnst(sp[X])));
      } else {
        nzz = G.axpb(nu, sp[Z], 0.0);
        nyz = G.axpb(G.ex(dn(dn(lnu, Y), Z)), std::max(sp[Y], sp[Z]), 0.0);
        nzx = G.axpb(G.ex(dn(dn(lnu, Z), X)), std::max(sp[Z], sp[X]), 0.0);
      }
    }
    int rxy = dens(dn(dn(lsrc, X), Y));
    int ryz = dens(dn(dn(lsrc, Y), Z));
    int rzx = dens(dn(dn(lsrc, Z), X));
    // Strain and stress, eq. (itv).  With the second-order switch
    // (do_2nddiv), a derivative along an axis flagged at the output's index
    // (|D2 ln rho| or |D2 ln e| of that cell above d2lnr_lim) is the two-point
    // difference: d6 + flag (d2 - d6).
    int flag[3] = {-1, -1, -1};
    if (p.do_2nddiv) {
      int lrr = G.lg(r), lee = G.lg(e);
      auto d2abs = [&](int f, int ax) {
        return G.ab(G.add(G.sub(G.shift(f, ax, 1), G.axpb(f, 2.0, 0.0)), G.shift(f, ax, -1)));
      };
      for (int a = 0; a < 3; ++a)
        flag[a] = G.stepf(G.maxi(d2abs(lrr, a), d2abs(lee, a)), p.d2lnr_lim);
    }
    auto sdup = [&](int f, int ax) {
      int d6 = ddup(f, ax);
      if (!p.do_2nddiv) return d6;
      int df = G.sub(G.shift(f, ax, 1), f);
      int d2 = (zs && ax == 2) ? G.mul(df, JC) : G.axpb(df, 1.0 / h[ax], 0.0);
      return G.add(d6, G.mul(flag[ax], G.sub(d2, d6)));
    };
    auto sddn = [&](int f, int ax) {
      int d6 = dddn(f, ax);
      if (!p.do_2nddiv) return d6;
      int df = G.sub(f, G.shift(f, ax, -1));
      int d2 = (zs && ax == 2) ? G.mul(df, JF) : G.axpb(df, 1.0 / h[ax], 0.0);
      return G.add(d6, G.mul(flag[ax], G.sub(d2, d6)));
    };
    int Sxx = sdup(u[X], X), Syy = sdup(u[Y], Y), Szz = sdup(u[Z], Z);
    int Sxy = G.axpb(G.add(sddn(u[X], Y), sddn(u[Y], X)), 0.5, 0.0);
    int Syz = G.axpb(G.add(sddn(u[Y], Z), sddn(u[Z], Y)), 0.5, 0.0);
    int Szx = G.axpb(G.add(sddn(u[Z], X), sddn(u[X], Z)), 0.5, 0.0);
    const int divs = p.do_2nddiv ? G.add(G.add(Sxx, Syy), Szz) : divu;
    auto diag = [&](int nii, int S) {
      int s = p.c1 != 0.0 ? G.add(S, G.axpb(divs, p.c1, 0.0)) : S;
      return G.mul(G.mul(r, nii), s);
    };
    txx = diag(nxx, Sxx);
    tyy = diag(nyy, Syy);
    tzz = diag(nzz, Szz);
    txy = G.mul(G.mul(rxy, nxy), Sxy);
    tyz = G.mul(G.mul(ryz, nyz), Syz);
    tzx = G.mul(G.mul(rzx, nzx), Szx);
    // Resistive field eta J with eta = nuB * nu of the edge.
    int Rx = G.mul(G.axpb(nyz, p.nuB, 0.0), Jx);
    int Ry = G.mul(G.axpb(nzx, p.nuB, 0.0), Jy);
    int Rz = G.mul(G.axpb(nxy, p.nuB, 0.0), Jz);
    if (p.do_quench) {
      // eq. (quench): one factor per component, over its differentiation axes;
      // |T| in the ratio is the 3-cell max of |T| along the axis.
      const double qe = p.quench_max3 ? -1.0 : p.quench_eps;
      auto quench = [&](int T, int a0, int a1) { return G.quench(T, a0, a1, p.qmax, p.qlim, qe); };
      txx = quench(txx, X, -1);
      tyy = quench(tyy, Y, -1);
      tzz = quench(tzz, Z, -1);
      txy = quench(txy, X, Y);
      tyz = quench(tyz, Y, Z);
      tzx = quench(tzx, Z, X);
      Rx = quench(Rx, Y, Z);
      Ry = quench(Ry, Z, X);
      Rz = quench(Rz, X, Y);
    }
    Ex = G.add(Ex, Rx);
    Ey = G.add(Ey, Ry);
    Ez = G.add(Ez, Rz);
    // eq. (vdiss) and Joule heating.
    int Qv = G.add(G.add(G.mul(txx, Sxx), G.mul(tyy, Syy)), G.mul(tzz, Szz));
    int off = G.add(G.add(up(up(G.mul(txy, Sxy), X), Y), up(up(G.mul(tyz, Syz), Y), Z)),
                    up(up(G.mul(tzx, Szx), Z), X));
    Qv = G.add(Qv, G.axpb(off, 2.0, 0.0));
    int Qj = G.add(G.add(up(up(G.mul(Rx, Jx), Y), Z), up(up(G.mul(Ry, Jy), Z), X)),
                   up(up(G.mul(Rz, Jz), X), Y));
    Q = G.add(Qv, Qj);
    // eq. (ediffuse): nuE ddup(dn(rho nu_ii) dddn e); with eq. (ediffav) (R23)
    // nuE ddup(dn(rho nu_ii) dn(e) dddn(ln e - ln <e>_h)), the log ratio as
    // log1p((ed - <ed>_h) / (e0 + <ed>_h)).
    int nii[3] = {nxx, nyy, nzz};
    int lrat = -1;
    if (p.ediffav) {
      const double e0 = r0 > 0 ? E0 / r0 : 0.0;
      const int pm = G.pmean(ed);
      lrat = G.lg1p(G.div(G.sub(ed, pm), G.axpb(pm, 1.0, e0)));
    }
    for (int d = 0; d < 3; ++d)
      ediff[d] = p.ediffav
          ? G.axpb(ddup(G.mul(dn(G.mul(r, nii[d]), d), G.mul(dn(e, d), dddn(lrat, d))), d), p.nuE, 0.0)
          : G.axpb(ddup(G.mul(dn(G.mul(r, nii[d]), d), dddn(ed, d)), d), p.nuE, 0.0);
  }

  // eq. (mass)
  int d_r = neg(G.add(G.add(ddup(pf[X], X), ddup(pf[Y], Y)), ddup(pf[Z], Z)));

  // eq. (mom): momentum flux components minus the (quenched) stress.
  auto minus_tau = [&](int flux, int tau) { return tau >= 0 ? G.sub(flux, tau) : flux; };
  auto Tdiag = [&](int d, int tau) {
    const int adv = G.mul(up(pf[d], d), up(u[d], d));
    return minus_tau(p.lnp_aver ? adv : G.add(adv, Pd), tau);
  };
  auto Toff = [&](int d, int a, int tau) {  // p_d carried along axis a
    return minus_tau(G.mul(dn(pf[d], a), dn(u[a], d)), tau);
  };
  auto grav = [&](int t, int d) {
    return p.g[d] != 0.0 ? G.add(t, G.axpb(rf[d], p.g[d], 0.0)) : t;
  };
  // eq. (pressure), lnp_aver (R24): P leaves the diagonal fluxes; its gradient
  // at the d face is exp(dn ln P_aver + dn lq) (dddn lq + dddn ln P_aver), lq =
  // ln(P/P_aver) = log1p((E' - <E'>_h) / (E0 + <E'>_h)); x and y derivatives of
  // the plane function ln P_aver vanish.
  int gradP[3] = {-1, -1, -1};
  if (p.lnp_aver) {
    const int pm = G.pmean(Ed);
    const int lpa = G.lg(G.axpb(pm, gm1, gm1 * E0));
    const int lq = G.lg1p(G.div(G.sub(Ed, pm), G.axpb(pm, 1.0, E0)));
    for (int d = 0; d < 3; ++d) {
      const int pface = G.ex(G.add(d == Z ? dn(lpa, Z) : lpa, dn(lq, d)));
      gradP[d] = G.mul(pface, d == Z ? G.add(dddn(lq, Z), dddn(lpa, Z)) : dddn(lq, d));
    }
  }
  int d_px = neg(dddn(Tdiag(X, txx), X));
  d_px = G.sub(d_px, ddup(Toff(X, Y, txy), Y));
  d_px = G.sub(d_px, ddup(Toff(X, Z, tzx), Z));
  d_px = G.add(d_px, up(G.mul(Jy, dn(B[Z], X)), Z));
  d_px = grav(G.sub(d_px, up(G.mul(Jz, dn(B[Y], X)), Y)), X);

  int d_py = neg(ddup(Toff(Y, X, txy), X));
  d_py = G.sub(d_py, dddn(Tdiag(Y, tyy), Y));
  d_py = G.sub(d_py, ddup(Toff(Y, Z, tyz), Z));
  d_py = G.add(d_py, up(G.mul(Jz, dn(B[X], Y)), X));
  d_py = grav(G.sub(d_py, up(G.mul(Jx, dn(B[Z], Y)), Z)), Y);

  int d_pz = neg(ddup(Toff(Z, X, tzx), X));
  d_pz = G.sub(d_pz, ddup(Toff(Z, Y, tyz), Y));
  d_pz = G.sub(d_pz, dddn(Tdiag(Z, tzz), Z));
  d_pz = G.add(d_pz, up(G.mul(Jx, dn(B[Y], Z)), Y));
  d_pz = grav(G.sub(d_pz, up(G.mul(Jy, dn(B[X], Z)), X)), Z);
  if (p.lnp_aver) {
    d_px = G.sub(d_px, gradP[X]);
    d_py = G.sub(d_py, gradP[Y]);
    d_pz = G.sub(d_pz, gradP[Z]);
  }

  // eq. (ien)
  int adv = G.add(G.add(ddup(G.mul(pf[X], dn(e, X)), X), ddup(G.mul(pf[Y], dn(e, Y)), Y)),
                  ddup(G.mul(pf[Z], dn(e, Z)), Z));
  int d_E = G.sub(neg(adv), G.mul(P, divu));
  if (Q >= 0) {
    d_E = G.add(d_E, Q);
    for (int d = 0; d < 3; ++d) d_E = G.add(d_E, ediff[d]);
  }
  if (p.t_cool > 0) {
    // Newtonian cooling, eqs. (NewtonCool), (rhocool): -rho (e - e_cool) / t_cool * f(rho).
    int qn = G.axpb(G.sub(E, G.axpb(r, p.e_cool, 0.0)), -1.0 / p.t_cool, 0.0);
    if (p.cool_cut) {
      int x = G.axpb(r, 1.0 / p.rho_cool, 0.0);
      int x2 = G.mul(x, x);
      int den = G.axpb(x2, 1.0, 1.0);
      int fac = p.cool_cut == 1 ? G.div(x2, den) : G.div(G.cnst(1.0), den);
      qn = G.mul(qn, fac);
    }
    d_E = G.add(d_E, qn);
  }
  if (p.t_chromo > 0) {
    // Chromospheric cooling, eq. (ChromoCool): -rho (rho/rho_bot)^(5/3) (e - <e>)/t,
    // <e> the horizontal-plane mean, taken on e - e0 (e0 cancels).
    int x53 = G.ex(G.axpb(G.lg(G.axpb(r, 1.0 / p.rho_bot, 0.0)), 5.0 / 3.0, 0.0));
    int de = G.sub(ed, G.pmean(ed));
    d_E = G.sub(d_E, G.mul(G.mul(r, x53), G.axpb(de, 1.0 / p.t_chromo, 0.0)));
  }
  if (p.cor_L0 > 0) {
    // Coronal thin cooling, eq. (CoronaCool): L0 T^(-1/2) rho^2 exp(-(T/1e4 K)^2),
    // T = Tunit (gamma - 1) e.
    int Tk = G.axpb(e, p.cor_Tunit * (p.gamma - 1.0), 0.0);
    int t4 = G.axpb(Tk, 1e-4, 0.0);
    int lam = G.mul(G.axpb(G.mul(r, r), p.cor_L0, 0.0),
                    G.div(G.ex(G.axpb(G.mul(t4, t4), -1.0, 0.0)), G.sq(Tk)));
    d_E = G.sub(d_E, lam);
  }

  // eq. (indu): dB/dt = -curl E.
  int d_Bx = neg(G.sub(ddup(Ez, Y), ddup(Ey, Z)));
  int d_By = neg(G.sub(ddup(Ex, Z), ddup(Ez, X)));
  int d_Bz = neg(G.sub(ddup(Ey, X), ddup(Ex, Y)));

  int outs[8] = {d_r, d_px, d_py, d_pz, d_E, d_Bx, d_By, d_Bz};
  for (int k = 0; k < 8; ++k) G.out[k] = outs[k];
  fuse_stencil_pairs(G);
}

// ---------------------------------------------------------------------------
// Executor
// ---------------------------------------------------------------------------
template <typename T>
int GraphExec<T>::init(const GraphDef& d, const Geo& g, bool with_grads) {
  release();
  def = d;
  geo = g;
  size_t nn = def.nodes.size();
  size_t nval = 0;
  for (auto& nd : def.nodes)
    if (nd.op != G_INPUT) ++nval;
  if (cudaMalloc(&vals, sizeof(T) * nval * g.n) != cudaSuccess) { vals = nullptr; return STAGGER_EOOM; }
  bool has_pmean = false, has_quench = false;
  for (auto& nd : def.nodes) {
    has_pmean |= nd.op == G_PMEAN;
    has_quench |= nd.op == G_QUENCH;
  }
  if (has_quench && with_grads &&
      cudaMalloc(&qscr, sizeof(T) * 7 * (size_t)g.n) != cudaSuccess) {
    qscr = nullptr;
    release();
    return STAGGER_EOOM;
  }
  if (has_pmean && cudaMalloc(&psum, sizeof(T) * g.nz) != cudaSuccess) {
    psum = nullptr;
    release();
    return STAGGER_EOOM;
  }
  if (!def.mesh.empty()) {
    std::vector<T> m(def.mesh.begin(), def.mesh.end());
    if (cudaMalloc(&mesh, sizeof(T) * m.size()) != cudaSuccess) {
      mesh = nullptr;
      release();
      return STAGGER_EOOM;
    }
    if (cudaMemcpy(mesh, m.data(), sizeof(T) * m.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      release();
      return STAGGER_ECUDA;
    }
  }
  if (with_grads) {
    if (cudaMalloc(&grads, sizeof(T) * nn * g.n) != cudaSuccess) {
      grads = nullptr;
      release();
      return STAGGER_EOOM;
    }
  }
  // Reverse-sweep bookkeeping: which nodes receive a gradient, and which
  // consumer slot gives each node its first contribution (in reverse order).
  hasg.assign(nn, 0);
  wa.assign(nn, 0);
  wb.assign(nn, 0);
  {
    std::vector<char> seen(nn, 0);
    for (int k = 0; k < 8; ++k) seen[def.out[k]] = hasg[def.out[k]] = 1;
    for (long long i = (long long)nn - 1; i >= 0; --i) {
      const GNode& nd = def.nodes[i];
      if (!hasg[i] || nd.op == G_INPUT || nd.op == G_CONST || nd.op == G_ZFIELD ||
          nd.op == G_STEP)
        continue;
      if (nd.a >= 0) { wa[i] = !seen[nd.a]; seen[nd.a] = hasg[nd.a] = 1; }
      if (nd.b >= 0) { wb[i] = !seen[nd.b]; seen[nd.b] = hasg[nd.b] = 1; }
    }
  }
  ptr.assign(nn, nullptr);
  size_t v = 0;
  for (size_t i = 0; i < nn; ++i)
    if (def.nodes[i].op != G_INPUT) ptr[i] = vals + (v++) * g.n;
  return STAGGER_OK;
}

template <typename T>
int GraphExec<T>::enable_concurrency() {
  if (nconc) return STAGGER_OK;
  for (int k = 0; k < GRAPH_NSTREAMS; ++k)
    if (cudaStreamCreateWithFlags(&aux[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&evjoin[k], cudaEventDisableTiming) != cudaSuccess)
      return STAGGER_ECUDA;
  if (cudaEventCreateWithFlags(&evfork, cudaEventDisableTiming) != cudaSuccess) return STAGGER_ECUDA;
  evn.assign(def.nodes.size(), nullptr);
  for (auto& e : evn)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return STAGGER_ECUDA;
  nconc = GRAPH_NSTREAMS;
  return STAGGER_OK;
}

template <typename T>
void GraphExec<T>::release() {
  for (auto e : evn)
    if (e) cudaEventDestroy(e);
  evn.clear();
  for (int k = 0; k < GRAPH_NSTREAMS; ++k) {
    if (aux[k]) cudaStreamDestroy(aux[k]);
    if (evjoin[k]) cudaEventDestroy(evjoin[k]);
    aux[k] = nullptr;
    evjoin[k] = nullptr;
  }
  if (evfork) cudaEventDestroy(evfork);
  evfork = nullptr;
  nconc = 0;
  if (vals) cudaFree(vals);
  if (grads) cudaFree(grads);
  if (mesh) cudaFree(mesh);
  if (psum) cudaFree(psum);
  if (qscr) cudaFree(qscr);
  vals = grads = mesh = psum = qscr = nullptr;
  ptr.clear();
}

static inline unsigned nblocks(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }
// z extent of the launch: GBZ * GZU cells per block along z (GZU per thread).
static inline dim3 ggrid(const Geo& g) {
  return dim3((unsigned)((g.nx + GBX - 1) / GBX), (unsigned)((g.ny + GBY - 1) / GBY),
              (unsigned)((g.nz + GBZ * GZU - 1) / (GBZ * GZU)));
}

// The forward and transpose kernel of each op (the op a template constant).
template <typename T>
using FwdK = void (*)(GNode, const T*, const T*, T*, const T*, Geo);
template <typename T>
using BwdK = void (*)(GNode, const T*, const T*, const T*, const T*, T*, T*, int, int, Geo);

template <typename T>
static FwdK<T> fwd_kernel(int op) {
  switch (op) {
    case G_STENCIL: return g_forward<T, G_STENCIL>;
    case G_SHIFT: return g_forward<T, G_SHIFT>;
    case G_STBIN: return g_forward<T, G_STBIN>;
    case G_STMUL: return g_forward<T, G_STMUL>;
    case G_ADD: return g_forward<T, G_ADD>;
    case G_SUB: return g_forward<T, G_SUB>;
    case G_MUL: return g_forward<T, G_MUL>;
    case G_DIV: return g_forward<T, G_DIV>;
    case G_MAX: return g_forward<T, G_MAX>;
    case G_EXP: return g_forward<T, G_EXP>;
    case G_LOG: return g_forward<T, G_LOG>;
    case G_LOG1P: return g_forward<T, G_LOG1P>;
    case G_SQRT: return g_forward<T, G_SQRT>;
    case G_ABS: return g_forward<T, G_ABS>;
    case G_AXPB: return g_forward<T, G_AXPB>;
    case G_CLAMPMIN: return g_forward<T, G_CLAMPMIN>;
    case G_CLAMPMAX: return g_forward<T, G_CLAMPMAX>;
    case G_STEP: return g_forward<T, G_STEP>;
    case G_ZFIELD: return g_forward<T, G_ZFIELD>;
    default: return g_forward<T, G_CONST>;
  }
}

template <typename T>
static BwdK<T> bwd_kernel(int op) {
  switch (op) {
    case G_STENCIL: return g_backward<T, G_STENCIL>;
    case G_SHIFT: return g_backward<T, G_SHIFT>;
    case G_STBIN: return g_backward<T, G_STBIN>;
    case G_STMUL: return g_backward<T, G_STMUL>;
    case G_ADD: return g_backward<T, G_ADD>;
    case G_SUB: return g_backward<T, G_SUB>;
    case G_MUL: return g_backward<T, G_MUL>;
    case G_DIV: return g_backward<T, G_DIV>;
    case G_MAX: return g_backward<T, G_MAX>;
    case G_EXP: return g_backward<T, G_EXP>;
    case G_LOG: return g_backward<T, G_LOG>;
    case G_LOG1P: return g_backward<T, G_LOG1P>;
    case G_SQRT: return g_backward<T, G_SQRT>;
    case G_ABS: return g_backward<T, G_ABS>;
    case G_AXPB: return g_backward<T, G_AXPB>;
    case G_CLAMPMIN: return g_backward<T, G_CLAMPMIN>;
    case G_CLAMPMAX: return g_backward<T, G_CLAMPMAX>;
    default: return g_backward<T, G_CONST>;   // no contribution
  }
}

// Fork the auxiliary streams from s (they then follow everything enqueued on
// s so far), and join them back into s.
template <typename T>
static int fork_streams(GraphExec<T>& G, cudaStream_t s) {
  STG_CUDA_OK(cudaEventRecord(G.evfork, s));
  for (int k = 0; k < G.nconc; ++k) STG_CUDA_OK(cudaStreamWaitEvent(G.aux[k], G.evfork, 0));
  return STAGGER_OK;
}
template <typename T>
static int join_streams(GraphExec<T>& G, cudaStream_t s) {
  for (int k = 0; k < G.nconc; ++k) {
    STG_CUDA_OK(cudaEventRecord(G.evjoin[k], G.aux[k]));
    STG_CUDA_OK(cudaStreamWaitEvent(s, G.evjoin[k], 0));
  }
  return STAGGER_OK;
}

template <typename T>
int GraphExec<T>::forward(T* const in[8], cudaStream_t s) {
  const size_t nn = def.nodes.size();
  for (size_t i = 0; i < nn; ++i)
    if (def.nodes[i].op == G_INPUT) ptr[i] = in[def.nodes[i].sk];
  const dim3 gg = ggrid(geo), gb(GBX, GBY, GBZ);
  // Concurrent form: the stream of each node (-1: an input, ready at the fork).
  std::vector<int> sto(nconc ? nn : 0, -1);
  int rr = 0, prev_scr = -1;
  if (nconc && fork_streams(*this, s)) return STAGGER_ECUDA;
  for (size_t i = 0; i < nn; ++i) {
    const GNode& nd = def.nodes[i];
    if (nd.op == G_INPUT) continue;
    const T* A = nd.a >= 0 ? ptr[nd.a] : nullptr;
    const T* B = nd.b >= 0 ? ptr[nd.b] : nullptr;
    cudaStream_t st = s;
    if (nconc) {
      // Follow the first operand's stream (chains stay on one stream); a node
      // without a computed operand starts the next stream in turn.
      int k = (nd.a >= 0 && sto[nd.a] >= 0) ? sto[nd.a]
            : (nd.b >= 0 && sto[nd.b] >= 0) ? sto[nd.b] : (rr++ % nconc);
      st = aux[k];
      for (int o : {nd.a, nd.b})
        if (o >= 0 && sto[o] >= 0 && sto[o] != k) STG_CUDA_OK(cudaStreamWaitEvent(st, evn[o], 0));
      if (nd.op == G_PMEAN && prev_scr >= 0 && sto[prev_scr] != k)
        STG_CUDA_OK(cudaStreamWaitEvent(st, evn[prev_scr], 0));   // psum is shared
      sto[i] = k;
    }
    if (nd.op == G_PMEAN) {
      g_plane_sum<T><<<geo.nz, 256, 0, st>>>(A, psum, geo);
      g_plane_bcast<T><<<gg, gb, 0, st>>>(psum, ptr[i], 0, geo);
      launches += 2;
      prev_scr = (int)i;
    } else if (nd.op == G_QUENCH) {
      g_quench_f<T><<<gg, gb, 0, st>>>(nd, A, ptr[i], geo);
      ++launches;
    } else {
      fwd_kernel<T>(nd.op)<<<gg, gb, 0, st>>>(nd, A, B, ptr[i], mesh, geo);
      ++launches;
    }
    if (nconc) STG_CUDA_OK(cudaEventRecord(evn[i], st));
  }
  if (nconc && join_streams(*this, s)) return STAGGER_ECUDA;
  STG_CUDA_OK(cudaGetLastError());
  return STAGGER_OK;
}

template <typename T>
int GraphExec<T>::backward(T* const seed[8], T* gin[8], cudaStream_t s) {
  if (!grads) return STAGGER_EINVAL;
  const size_t nn = def.nodes.size();
  const int bs = 256;
  const dim3 gg = ggrid(geo), gb(GBX, GBY, GBZ);
  // Seeds are the first contribution to the outputs' gradients: copy them.
  for (int k = 0; k < 8; ++k)
    STG_CUDA_OK(cudaMemcpyAsync(grads + (size_t)def.out[k] * geo.n, seed[k],
                                sizeof(T) * geo.n, cudaMemcpyDeviceToDevice, s));
  // Concurrent form: the last launch that wrote each gradient array (-1: none
  // since the fork), and its stream.
  std::vector<int> lastw(nconc ? nn : 0, -1), sto(nconc ? nn : 0, -1);
  int rr = 0, prev_scr = -1;
  if (nconc && fork_streams(*this, s)) return STAGGER_ECUDA;
  for (long long i = (long long)nn - 1; i >= 0; --i) {
    const GNode& nd = def.nodes[i];
    if (!hasg[i] || nd.op == G_INPUT || nd.op == G_CONST || nd.op == G_ZFIELD ||
        nd.op == G_STEP)
      continue;
    const T* A = nd.a >= 0 ? ptr[nd.a] : nullptr;
    const T* B = nd.b >= 0 ? ptr[nd.b] : nullptr;
    T* gA = nd.a >= 0 ? grads + (size_t)nd.a * geo.n : nullptr;
    T* gB = nd.b >= 0 ? grads + (size_t)nd.b * geo.n : nullptr;
    cudaStream_t st = s;
    if (nconc) {
      // Wait for the complete gradient of this node, for the previous writer
      // of each gradient it adds to, and for the previous user of the shared
      // scratch (quench, plane mean).
      const int own = lastw[i];
      int k = own >= 0 ? sto[own] : (rr++ % nconc);
      st = aux[k];
      const bool scr = nd.op == G_QUENCH || nd.op == G_PMEAN;
      for (int w : {own, nd.a >= 0 ? lastw[nd.a] : -1, nd.b >= 0 ? lastw[nd.b] : -1,
                    scr ? prev_scr : -1})
        if (w >= 0 && sto[w] != k) STG_CUDA_OK(cudaStreamWaitEvent(st, evn[w], 0));
      sto[i] = k;
      if (scr) prev_scr = (int)i;
    }
    if (nd.op == G_PMEAN) {
      g_plane_sum<T><<<geo.nz, 256, 0, st>>>(grads + (size_t)i * geo.n, psum, geo);
      g_plane_bcast<T><<<gg, gb, 0, st>>>(psum, gA, wa[i] ? 0 : 1, geo);
      launches += 2;
    } else if (nd.op == G_QUENCH) {
      g_quench_b1<T><<<gg, gb, 0, st>>>(nd, A, grads + (size_t)i * geo.n, qscr, geo);
      g_quench_b3<T><<<gg, gb, 0, st>>>(nd, A, qscr, gA, wa[i], geo);
      launches += 2;
    } else {
      bwd_kernel<T>(nd.op)<<<gg, gb, 0, st>>>(nd, A, B, ptr[i], grads + (size_t)i * geo.n, gA,
                                              gB, wa[i], wb[i], geo);
      ++launches;
    }
    if (nconc) {
      STG_CUDA_OK(cudaEventRecord(evn[i], st));
      if (nd.a >= 0) lastw[nd.a] = (int)i;
      if (nd.b >= 0) lastw[nd.b] = (int)i;
    }
  }
  if (nconc && join_streams(*this, s)) return STAGGER_ECUDA;
  for (int k = 0; k < 8; ++k) {
    if (!hasg[def.in[k]]) continue;   // the outputs do not depend on this input
    g_add_into<T><<<nblocks(geo.n, bs), bs, 0, s>>>(gin[k], grads + (size_t)def.in[k] * geo.n, geo.n);
    ++launches;
  }
  STG_CUDA_OK(cudaGetLastError());
  return STAGGER_OK;
}

template struct GraphExec<float>;
template struct GraphExec<double>;

}  // namespace stg
