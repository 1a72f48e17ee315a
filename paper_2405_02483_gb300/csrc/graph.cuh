// Op graph of the MHD right-hand side: the equations written as a DAG of
// primitive staggered operations (6th-order derivatives, 5th-order
// interpolations, shifts, pointwise arithmetic).  Each primitive has a forward
// CUDA kernel and a hand-written transpose (vector-Jacobian) kernel, so the
// graph gives an unfused forward and, swept in reverse, the adjoint.
#pragma once

#include <map>
#include <tuple>
#include <utility>
#include <vector>

#include "common.cuh"

namespace stg {

enum GOp {
  G_INPUT = 0, G_STENCIL, G_SHIFT, G_ADD, G_SUB, G_MUL, G_DIV, G_MAX,
  G_EXP, G_LOG, G_LOG1P, G_SQRT, G_ABS, G_AXPB, G_CLAMPMIN, G_CLAMPMAX, G_CONST,
  G_STEP,  // 1 where a > c0, else 0 (a switch: no gradient)
  G_ZFIELD, // a mesh array over z (sk: 0 1/dz_c, 1 1/dz_f, 2 dz_c, 3 dz_f, 4 local dl_min)
  G_PMEAN,  // mean of a over the horizontal plane (constant z) of each cell
  G_QUENCH, // eq. (quench) of a over axes axis and sk (-1: one axis); c0 qmax, c1 qlim, c2 eps
  // Fused pairs (formed after the build, see fuse_stencil_pairs): a stencil
  // (kind sk, axis, spacing c0) of a combined with b by iop (G_ADD, G_SUB,
  // G_MUL; side 1: b comes first), and a stencil of the product a b.
  G_STBIN,
  G_STMUL,
  // The sum or difference (iop) of two stencils: (kind sk, axis, spacing c0)
  // of a and (kind sk2, axis2, spacing h2) of b.
  G_ST2,
  // exp of a stencil (kind sk, axis, spacing c0) of a.
  G_STEXP,
  // Three neighbours along axis combined by iop (G_ADD or G_MAX) as the graph
  // built them: (a(i + sk) op a(i)) op a(i - sk).
  G_NB3
};
enum GStencil { ST_UP = 0, ST_DN, ST_DDUP, ST_DDDN };

struct GNode {
  int op;       // GOp
  int a, b;     // input node ids (-1 if unused)
  int axis;     // 0 = x, 1 = y, 2 = z (stencil / shift)
  int sk;       // GStencil kind, or shift distance
  double c0, c1;  // scalars: spacing h (derivative), a*x+b, clamp bound, const
  double c2 = 0;  // G_QUENCH: weight of max3|T| added to |T| (< 0: max3|T| alone)
  int iop = 0;    // G_STBIN: the binary op
  int side = 0;   // G_STBIN: 1 when the stencil is the second operand
  double ps = 1, pt = 0;  // epilogue: the node's value is ps v + pt (a folded G_AXPB)
  int axis2 = 0, sk2 = 0;  // G_ST2: the second stencil
  double h2 = 0;
  // A folded sum: the node's value v becomes v + C (pop 1), v - C (2) or
  // C - v (3), C the value of node c; the epilogue (ps, pt) applies after it.
  int c = -1, pop = 0;
  // Float copies of the constants, for the FP32 kernels, and whether the
  // epilogue is other than the identity (set when the graph is complete).
  float f0 = 0, f1 = 0, f2 = 0, fh2 = 0, fps = 1, fpt = 0;
  int ep = 0;
};

// Precision-independent description of the graph.
struct GraphDef {
  std::vector<GNode> nodes;
  int in[8];    // input node per state field (stored deviation)
  int out[8];   // output node per time derivative

  // Every node is a pure function of its inputs and constants, so a node
  // identical to an earlier one (commutative inputs in either order) is that
  // node: the graph holds each distinct value once.  The quench node takes its
  // eps after the push and is never shared.
  int push(int op, int a, int b, int axis, int sk, double c0, double c1) {
    if (op != G_INPUT && op != G_QUENCH) {
      if ((op == G_ADD || op == G_MUL || op == G_MAX) && a > b) std::swap(a, b);
      const auto key = std::make_tuple(op, a, b, axis, sk, c0, c1);
      const auto it = memo.find(key);
      if (it != memo.end()) return it->second;
      memo[key] = (int)nodes.size();
    }
    GNode n{op, a, b, axis, sk, c0, c1};
    nodes.push_back(n);
    return (int)nodes.size() - 1;
  }
  std::map<std::tuple<int, int, int, int, int, double, double>, int> memo;
  int input(int k) { return in[k] = push(G_INPUT, -1, -1, 0, k, 0, 0); }
  int st(int kind, int a, int axis, double h) { return push(G_STENCIL, a, -1, axis, kind, h, 0); }
  int up(int a, int ax) { return st(ST_UP, a, ax, 1.0); }
  int dn(int a, int ax) { return st(ST_DN, a, ax, 1.0); }
  int shift(int a, int ax, int s) { return push(G_SHIFT, a, -1, ax, s, 0, 0); }
  int add(int a, int b) { return push(G_ADD, a, b, 0, 0, 0, 0); }
  int sub(int a, int b) { return push(G_SUB, a, b, 0, 0, 0, 0); }
  int mul(int a, int b) { return push(G_MUL, a, b, 0, 0, 0, 0); }
  int div(int a, int b) { return push(G_DIV, a, b, 0, 0, 0, 0); }
  int maxi(int a, int b) { return push(G_MAX, a, b, 0, 0, 0, 0); }
  int ex(int a) { return push(G_EXP, a, -1, 0, 0, 0, 0); }
  int lg(int a) { return push(G_LOG, a, -1, 0, 0, 0, 0); }
  int lg1p(int a) { return push(G_LOG1P, a, -1, 0, 0, 0, 0); }
  int sq(int a) { return push(G_SQRT, a, -1, 0, 0, 0, 0); }
  int ab(int a) { return push(G_ABS, a, -1, 0, 0, 0, 0); }
  int axpb(int a, double s, double t) { return push(G_AXPB, a, -1, 0, 0, s, t); }
  int cmin(int a, double c) { return push(G_CLAMPMIN, a, -1, 0, 0, c, 0); }
  int cmax(int a, double c) { return push(G_CLAMPMAX, a, -1, 0, 0, c, 0); }
  int cnst(double c) { return push(G_CONST, -1, -1, 0, 0, c, 0); }
  int stepf(int a, double c) { return push(G_STEP, a, -1, 0, 0, c, 0); }
  int zfield(int which) { return push(G_ZFIELD, -1, -1, 2, which, 0, 0); }
  int pmean(int a) { return push(G_PMEAN, a, -1, 0, 0, 0, 0); }
  int quench(int a, int a0, int a1, double qmax, double qlim, double eps) {
    const int id = push(G_QUENCH, a, -1, a0, a1, qmax, qlim);
    nodes[id].c2 = eps;
    return id;
  }
  // Stretched z mesh: the five arrays of G_ZFIELD, nz values each (empty when uniform).
  std::vector<double> mesh;
};

// Build the right-hand-side graph for a grid and parameter set; with fuse,
// merge single-use nodes into their consumers (the same values, fewer arrays
// and launches), without it keep one node per primitive.
void build_rhs_graph(GraphDef& G, const stagger_grid& grid, const stagger_params& p,
                     bool fuse = true);

// The reverse sweep's plan, from the graph alone: which nodes receive a
// gradient (hasg), which operand slot of a node gives an input its first
// contribution and so writes rather than adds (wa, wb, wc), and the gradient
// array of each node.  A gradient is live from its first contribution (by its
// highest-numbered consumer) to its own transpose; arrays are reused once the
// transpose that read them has run: gslot[i] is node i's array (-1: none),
// gprev[i] the node whose transpose last read that array before (-1: a fresh
// array), which the first writer must wait for.  Returns the number of arrays.
struct ReversePlan {
  std::vector<char> hasg, wa, wb, wc;
  std::vector<int> gslot, gprev;
  int nslots = 0;
};
void plan_reverse(const GraphDef& G, ReversePlan& P);
// Whether node op has a transpose kernel (the others pass no gradient on).
inline bool has_transpose(int op) {
  return op != G_INPUT && op != G_CONST && op != G_ZFIELD && op != G_STEP;
}

#ifndef GRAPH_NSTREAMS
#define GRAPH_NSTREAMS 4
#endif

// Device executor for one precision.  Holds one value and one gradient array
// of n cells per node (inputs point at caller memory and need none).
template <typename T>
struct GraphExec {
  GraphDef def;
  Geo geo;
  T* vals = nullptr;     // node values (non-input nodes)
  T* mesh = nullptr;     // the mesh arrays of G_ZFIELD on the device, or null
  T* psum = nullptr;     // per-plane sums of G_PMEAN (nz), or null
  T* qscr = nullptr;     // 15 arrays of scratch for the G_QUENCH transpose, or null
  T* grads = nullptr;    // gradient arrays (rp.nslots, reused by liveness)
  std::vector<T*> ptr;   // value pointer per node
  ReversePlan rp;        // the reverse sweep's gradient flags and arrays
  T* gptr(int i) { return grads + (size_t)rp.gslot[i] * geo.n; }
  long long launches = 0;
  // Concurrent sweeps: with nconc auxiliary streams each node's launch waits
  // only on the launches it depends on (its operands' values in the forward;
  // its own gradient and the previous writer of each gradient it adds to in
  // the reverse; the previous user of the shared quench and plane-mean
  // scratch), so a sweep captured into a CUDA graph becomes a DAG whose
  // independent kernels overlap.  0: one stream, in node order.
  int nconc = 0;
  cudaStream_t aux[GRAPH_NSTREAMS] = {};
  std::vector<cudaEvent_t> evn;
  cudaEvent_t evfork = nullptr, evjoin[GRAPH_NSTREAMS] = {};
  int enable_concurrency();

  int init(const GraphDef& d, const Geo& g, bool with_grads);
  void release();
  // Evaluate every node; inputs are the 8 stored deviation arrays.
  int forward(T* const in[8], cudaStream_t s);
  // Reverse sweep: seed the 8 output gradients, accumulate into gin[8]
  // (+=).  forward() must have run on the same inputs.
  int backward(T* const seed[8], T* gin[8], cudaStream_t s);
  T* output(int k) { return ptr[def.out[k]]; }
};

}  // namespace stg
