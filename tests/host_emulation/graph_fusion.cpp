// Host build of the op graph: the graph with its merged nodes (fused stencil
// pairs, stencil sums and exps, 3-cell maxima and sums, folded sums and
// scalings), swept by the one-cell and by the four-x-cell kernels, against
// the graph of one node per primitive, the kernels run over their launch
// grids one thread at a time.  The forward outputs must be equal bit for bit; the reverse
// sweep's input gradients may differ only by rounding (the merged transposes
// scale a gathered cotangent instead of gathering a scaled one): within 1e-12
// (FP64) or 1e-5 (FP32) of each field's largest gradient.  Cases: the
// benchmark's viscosity and quench (also on a state uniform along z, whose
// maxima along z tie exactly); with chromospheric and coronal cooling (plane
// means, exp, sqrt); Smagorinsky with the bulk term, gravity, ediffav,
// ln(P/P_aver), the second-order switch and no log interpolation on a
// stretched z mesh.  Exit status: the number of failing (case, precision)
// pairs.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
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
#include "../../paper_2405_02483_gb300/csrc/graph_kernels.cuh"
#include "../../paper_2405_02483_gb300/csrc/graph_build.cu"
using namespace stg;

static long long g_four = 0;   // four-x-cell launches run

template <class K>
static void run(const Geo& g, K kern, bool four = false) {
  g_four += four;
  const dim3 bd(GBX, GBY, GBZ);
  const dim3 gd(four ? (g.nx / 4 + GBX - 1) / GBX : (g.nx + GBX - 1) / GBX, (g.ny + GBY - 1) / GBY,
                four ? (g.nz + GBZ - 1) / GBZ : (g.nz + GBZ * GZU - 1) / (GBZ * GZU));
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

// A flat launch (the pointwise kernels): blocks of 256 threads, grid-stride.
template <class K>
static void run1d(long long work, K kern) {
  const unsigned nb = (unsigned)std::min<long long>((work + 255) / 256, 8192);
  gridDim = dim3(nb, 1, 1);
  blockDim = dim3(256, 1, 1);
  for (unsigned b = 0; b < nb; ++b)
    for (unsigned t = 0; t < 256; ++t) {
      blockIdx = make_uint3(b, 0, 0);
      threadIdx = make_uint3(t, 0, 0);
      kern();
    }
}
static bool al16(const void* p) { return ((uintptr_t)p & 15) == 0; }

// The executor's sweeps (graph.cu) on the host, one node after another.
template <typename T>
struct HostExec {
  GraphDef d;
  Geo g;
  bool allow4 = true;   // the four-x-cell kernels where the executor takes them
  std::vector<std::vector<T>> v, gr;   // node values; the plan's gradient arrays
  std::vector<T> mesh;
  ReversePlan rp;
  int nslots = 0;

  void init() {
    const size_t nn = d.nodes.size();
    v.assign(nn, std::vector<T>(g.n, 0));
    mesh.assign(d.mesh.begin(), d.mesh.end());
    plan_reverse(d, rp);
    // NaN-filled: a contribution added to an array that its first writer
    // did not write (a fresh or a reused one) shows as non-finite.
    gr.assign(rp.nslots, std::vector<T>(g.n, (T)NAN));
  }
  T* gp(int x) { return gr[rp.gslot[x]].data(); }
  // The horizontal-plane mean, written or added (G_PMEAN and its transpose).
  void pmean(const T* a, T* o, bool add) const {
    for (int k = 0; k < g.nz; ++k) {
      T s = 0;
      for (long long q = 0; q < g.sz; ++q) s += a[k * g.sz + q];
      s /= (T)g.sz;
      for (long long q = 0; q < g.sz; ++q) o[k * g.sz + q] = add ? o[k * g.sz + q] + s : s;
    }
  }
  void forward(const std::vector<std::vector<T>>& in) {
    const T* M = mesh.empty() ? nullptr : mesh.data();
    for (size_t i = 0; i < d.nodes.size(); ++i) {
      const GNode nd = d.nodes[i];
      if (nd.op == G_INPUT) {
        v[i] = in[nd.sk];
        continue;
      }
      const T* A = nd.a >= 0 ? v[nd.a].data() : nullptr;
      const T* B = nd.b >= 0 ? v[nd.b].data() : nullptr;
      const T* C = nd.c >= 0 ? v[nd.c].data() : nullptr;
      T* out = v[i].data();
      const Geo& G = g;
      const int vec = g.n % 4 == 0 && al16(A) && al16(B) && al16(C) && al16(out);
      const bool four = allow4 && g.nx % 4 == 0 && al16(A) && al16(B) && al16(C) && al16(out) &&
                        ((nd.op != G_SHIFT && nd.op != G_NB3) || nd.sk == 1 || nd.sk == -1);
#define FW(OP)                                                                    \
  case OP:                                                                        \
    if (four)                                                                     \
      run(G, [&] { g_forward4<T, OP>(nd, A, B, C, out, M, G); }, true);           \
    else                                                                          \
      run(G, [&] { g_forward<T, OP>(nd, A, B, C, out, M, G); });                  \
    break;
#define FP(OP)                                                                         \
  case OP:                                                                             \
    run1d(vec ? g.n / 4 : g.n, [&] { g_forward_pw<T, OP>(nd, A, B, C, out, g.n, vec); }); \
    break;
      switch (nd.op) {
        case G_PMEAN: pmean(A, out, false); break;
        case G_QUENCH:
          if (allow4 && g.nx % 4 == 0 && al16(A) && al16(out))
            run(G, [&] { g_quench_f4<T>(nd, A, out, G); }, true);
          else
            run(G, [&] { g_quench_f<T>(nd, A, out, G); });
          break;
        FW(G_STENCIL) FW(G_SHIFT) FW(G_STBIN) FW(G_STMUL) FW(G_ST2) FW(G_STEXP) FW(G_NB3)
        FW(G_ZFIELD) FP(G_ADD) FP(G_SUB) FP(G_MUL) FP(G_DIV) FP(G_MAX) FP(G_EXP) FP(G_LOG)
        FP(G_LOG1P) FP(G_SQRT) FP(G_ABS) FP(G_AXPB) FP(G_CLAMPMIN) FP(G_CLAMPMAX) FP(G_STEP)
        FP(G_CONST)
        default: printf("no forward for op %d\n", nd.op); exit(100);
      }
#undef FW
#undef FP
    }
  }
  void backward(const std::vector<std::vector<T>>& seed, std::vector<std::vector<T>>& gin) {
    for (int k = 0; k < 8; ++k) gr[rp.gslot[d.out[k]]] = seed[k];
    std::vector<T> S(15 * g.n);
    for (long long i = (long long)d.nodes.size() - 1; i >= 0; --i) {
      const GNode nd = d.nodes[i];
      if (!rp.hasg[i] || !has_transpose(nd.op)) continue;
      const T* A = nd.a >= 0 ? v[nd.a].data() : nullptr;
      const T* B = nd.b >= 0 ? v[nd.b].data() : nullptr;
      T* gA = nd.a >= 0 ? gp(nd.a) : nullptr;
      T* gB = nd.b >= 0 ? gp(nd.b) : nullptr;
      T* gC = nd.c >= 0 ? gp(nd.c) : nullptr;
      const T* out = v[i].data();
      const T* go = gp((int)i);
      const int WA = rp.wa[i], WB = rp.wb[i], WC = rp.wc[i];
      const Geo& G = g;
      const int vec = g.n % 4 == 0 && al16(A) && al16(B) && al16(out) && al16(go) && al16(gA) &&
                      al16(gB) && al16(gC);
      const bool four = allow4 && g.nx % 4 == 0 && vec &&
                        ((nd.op != G_SHIFT && nd.op != G_NB3) || nd.sk == 1 || nd.sk == -1);
#define BW(OP)                                                                                 \
  case OP:                                                                                     \
    if (four)                                                                                  \
      run(G, [&] { g_backward4<T, OP>(nd, A, B, out, go, gA, gB, gC, WA, WB, WC, G); }, true); \
    else                                                                                       \
      run(G, [&] { g_backward<T, OP>(nd, A, B, out, go, gA, gB, gC, WA, WB, WC, G); });        \
    break;
#define BP(OP)                                                                                 \
  case OP:                                                                                     \
    run1d(vec ? g.n / 4 : g.n,                                                                 \
          [&] { g_backward_pw<T, OP>(nd, A, B, out, go, gA, gB, gC, WA, WB, WC, g.n, vec); }); \
    break;
      switch (nd.op) {
        case G_PMEAN: pmean(go, gA, !WA); break;
        case G_QUENCH:
          if (allow4 && g.nx % 4 == 0 && al16(A) && al16(go) && al16(gA) && al16(S.data())) {
            run(G, [&] { g_quench_q4<T>(nd, A, S.data() + 7 * G.n, G); }, true);
            run(G, [&] { g_quench_b1_4<T>(nd, A, S.data() + 7 * G.n, go, S.data(), G); }, true);
            run(G, [&] { g_quench_b3_4<T>(nd, S.data() + 7 * G.n, S.data(), gA, WA, G); }, true);
          } else {
            run(G, [&] { g_quench_q<T>(nd, A, S.data() + 7 * G.n, G); });
            run(G, [&] { g_quench_b1<T>(nd, A, S.data() + 7 * G.n, go, S.data(), G); });
            run(G, [&] { g_quench_b3<T>(nd, S.data() + 7 * G.n, S.data(), gA, WA, G); });
          }
          break;
        BW(G_STENCIL) BW(G_SHIFT) BW(G_STBIN) BW(G_STMUL) BW(G_ST2) BW(G_STEXP) BW(G_NB3)
        BP(G_ADD) BP(G_SUB) BP(G_MUL) BP(G_DIV) BP(G_MAX) BP(G_EXP) BP(G_LOG) BP(G_LOG1P)
        BP(G_SQRT) BP(G_ABS) BP(G_AXPB) BP(G_CLAMPMIN) BP(G_CLAMPMAX)
        default: printf("no transpose for op %d\n", nd.op); exit(100);
      }
#undef BW
#undef BP
    }
    for (int k = 0; k < 8; ++k)
      gin[k] = rp.gslot[d.in[k]] >= 0 ? gr[rp.gslot[d.in[k]]] : std::vector<T>(g.n, (T)0);
    nslots = rp.nslots;
  }
};

// The library's defaults (stagger_params_default), for the fields the graph reads.
static stagger_params base_params() {
  stagger_params p;
  memset(&p, 0, sizeof(p));
  p.gamma = 5.0 / 3.0;
  p.nuE = p.nuB = 1.0;
  p.qmax = 8.0;
  p.qlim = 2.0;
  p.quench_eps = 1e-4;
  p.log_interp = 1;
  p.rho_cool = 1.0;
  p.d2lnr_lim = 0.3;
  p.rho_bot = 1.0;
  p.cor_Tunit = 1.0;
  p.nu1 = 0.04;
  p.nu2 = 1.0;
  p.nu3 = 0.04;
  p.do_quench = 1;
  p.ref[0] = 1.0;
  p.ref[4] = 1.5;
  p.ref[7] = 0.5;
  return p;
}

// zuni: every input field uniform along z, so that the 3-cell maxima along z
// meet exact ties (split evenly by the transposes).
// Three sweeps of the same state: one node per primitive with one-cell
// kernels (the reference), the merged graph with one-cell kernels, and the
// merged graph with the four-x-cell kernels where they apply.  zuni: every
// input field uniform along z, so that the 3-cell maxima along z meet exact
// ties (split evenly by the transposes).
template <typename T>
static int compare(const char* name, const stagger_grid& gg, const stagger_params& p, double tol,
                   bool zuni = false) {
  const Geo g = make_geo(gg.nx, gg.ny, gg.nz);
  std::mt19937_64 rng(7);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  std::vector<std::vector<T>> in(8, std::vector<T>(g.n)), seed(8, std::vector<T>(g.n));
  for (int k = 0; k < 8; ++k)
    for (auto& x : in[k]) x = (T)((k == 0 || k == 4 ? 0.1 : 0.3) * U(rng));
  if (zuni)
    for (int k = 0; k < 8; ++k)
      for (long long q = g.sz; q < g.n; ++q) in[k][q] = in[k][q % g.sz];
  for (int k = 0; k < 8; ++k)
    for (auto& x : seed[k]) x = (T)U(rng);
  std::vector<std::vector<T>> res[3], gin[3];
  size_t nodes[3];
  long long four[3];
  int arrays[3];
  for (int t = 0; t < 3; ++t) {
    g_four = 0;
    HostExec<T> h;
    h.g = g;
    h.allow4 = t == 2;
    build_rhs_graph(h.d, gg, p, t > 0);
    nodes[t] = h.d.nodes.size();
    h.init();
    h.forward(in);
    for (int k = 0; k < 8; ++k) res[t].push_back(h.v[h.d.out[k]]);
    gin[t].resize(8);
    h.backward(seed, gin[t]);
    four[t] = g_four;
    arrays[t] = h.nslots;
  }
  int fails = 0;
  for (int t = 1; t < 3; ++t) {
    long long diff = 0, bad = 0;
    double worst = 0;
    for (int k = 0; k < 8; ++k) {
      double e = 0, s = 0;
      for (long long q = 0; q < g.n; ++q) {
        if (std::memcmp(&res[0][k][q], &res[t][k][q], sizeof(T)) != 0) ++diff;
        if (!std::isfinite((double)res[t][k][q]) || !std::isfinite((double)gin[t][k][q])) ++bad;
        e = std::max(e, std::fabs((double)gin[0][k][q] - (double)gin[t][k][q]));
        s = std::max(s, std::fabs((double)gin[0][k][q]));
      }
      worst = std::max(worst, e / std::max(s, 1e-300));
    }
    const bool ok = diff == 0 && bad == 0 && worst <= tol;
    printf("%s %s %s (%lld four-cell launches): %zu -> %zu nodes, %d -> %d gradient arrays, "
           "forward %lld differing values, %lld non-finite, reverse max rel err %.2e%s\n", name,
           sizeof(T) == 8 ? "FP64" : "FP32", t == 1 ? "one-cell" : "four-cell", four[t],
           nodes[0], nodes[t], arrays[0], arrays[t], diff, bad, worst, ok ? "" : "  FAIL");
    fails += !ok;
  }
  return fails;
}

int main() {
  int fails = 0;
  const stagger_grid g1 = {16, 11, 9, 1.0 / 16, 1.0 / 11, 1.0 / 9};
  const stagger_grid g3 = {13, 11, 9, 1.0 / 13, 1.0 / 11, 1.0 / 9};   // no four-cell kernels
  stagger_params visc = base_params();
  stagger_params cool = base_params();
  cool.t_chromo = 0.05;
  cool.rho_bot = 0.9;
  cool.cor_L0 = 0.3;
  cool.cor_Tunit = 8e3;
  cool.t_cool = 0.2;
  cool.e_cool = 1.2;
  // A stretched z mesh: centre and face spacings of a smooth mapping.
  const stagger_grid g2 = {12, 10, 11, 1.0 / 12, 1.0 / 10, 1.0 / 11};
  std::vector<double> zc(g2.nz), zf(g2.nz);
  for (int k = 0; k < g2.nz; ++k) {
    zc[k] = (1.0 + 0.3 * std::sin(2 * M_PI * (k + 0.5) / g2.nz)) / g2.nz;
    zf[k] = (1.0 + 0.3 * std::sin(2 * M_PI * k / (double)g2.nz)) / g2.nz;
  }
  stagger_params opts = base_params();
  opts.csmag = 0.2;
  opts.c1 = -1.0 / 3.0;
  opts.g[0] = 0.1;
  opts.g[2] = -1.0;
  opts.ediffav = 1;
  opts.lnp_aver = 1;
  opts.do_2nddiv = 1;
  opts.log_interp = 0;
  opts.zc = zc.data();
  opts.zf = zf.data();
  fails += compare<double>("viscosity+quench", g1, visc, 1e-12);
  fails += compare<float>("viscosity+quench", g1, visc, 1e-5);
  fails += compare<double>("viscosity+quench z-uniform", g1, visc, 1e-12, true);
  fails += compare<float>("viscosity+quench z-uniform", g1, visc, 1e-5, true);
  fails += compare<double>("cooling", g3, cool, 1e-12);
  fails += compare<float>("cooling", g3, cool, 1e-5);
  fails += compare<double>("options+stretched", g2, opts, 1e-12);
  fails += compare<float>("options+stretched", g2, opts, 1e-5);
  return fails;
}
