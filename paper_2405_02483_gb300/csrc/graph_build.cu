// The right-hand-side op graph (see graph.cuh): its construction from the
// equations and the passes that merge nodes.  Host code only.
#include <math.h>

#include <algorithm>
#include <vector>

#include "graph.cuh"

namespace stg {

// ---------------------------------------------------------------------------
// The right-hand side, eqs. (mass), (mom), (itv), (ien), (vdiss), (indu),
// (ohm), written on the stored deviations f' (full value ref + f').
// ---------------------------------------------------------------------------
// Every node is a whole-array pass whose launch, ramp and tail cost as much as
// its bytes, so a stencil that feeds one sum, difference, product or exp, two
// stencils that feed one sum or difference, and a product that feeds one
// stencil are merged into one node (G_STBIN, G_ST2, G_STEXP, G_STMUL): the
// pair's intermediate array and launches go away, and the fused node's
// transpose is the pair's (the stencil's gather-form transpose of the
// cotangent, times the other factor where there is one).  A node used twice,
// or as an output, keeps its array.  (A quench that reads the product forming
// its T at every tap measured slower than the product's own node: its many
// taps then load two arrays.)  The graph is then compacted.
static void compact(GraphDef& G, const std::vector<char>& dead);
static bool generic_op(int op);

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
    auto lone_st = [&](int src) {
      return src >= 0 && !dead[src] && G.nodes[src].op == G_STENCIL && uses[src] == 1;
    };
    if ((nd.op == G_ADD || nd.op == G_SUB) && lone_st(nd.a) && lone_st(nd.b) && nd.a != nd.b) {
      const GNode s1 = G.nodes[nd.a], s2 = G.nodes[nd.b];
      dead[nd.a] = dead[nd.b] = 1;
      GNode f = nd;
      f.op = G_ST2;
      f.iop = nd.op;
      f.a = s1.a;
      f.b = s2.a;
      f.axis = s1.axis;
      f.sk = s1.sk;
      f.c0 = s1.c0;
      f.c1 = 0;
      f.axis2 = s2.axis;
      f.sk2 = s2.sk;
      f.h2 = s2.c0;
      nd = f;
    } else if (nd.op == G_ADD || nd.op == G_SUB || nd.op == G_MUL) {
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
    } else if (nd.op == G_EXP && lone_st(nd.a)) {
      const GNode st = G.nodes[nd.a];
      dead[nd.a] = 1;
      nd.op = G_STEXP;
      nd.a = st.a;
      nd.axis = st.axis;
      nd.sk = st.sk;
      nd.c0 = st.c0;
    } else if (nd.op == G_STENCIL && nd.a >= 0 && !dead[nd.a] && G.nodes[nd.a].op == G_MUL &&
               uses[nd.a] == 1) {
      const GNode m = G.nodes[nd.a];
      dead[nd.a] = 1;
      nd.op = G_STMUL;
      nd.a = m.a;
      nd.b = m.b;
    }
  }
  compact(G, dead);
}

// A scaling c0 x + c1 (G_AXPB) whose operand feeds nothing else becomes that
// operand's epilogue (ps, pt): one array and one launch per sweep fewer.  The
// operand's transpose then takes ps times the cotangent (every transpose is
// linear in it).  Exp and sqrt stay apart (their transposes read their own
// value), and so do the nodes with their own kernels or without a gradient.
static void fold_affine(GraphDef& G) {
  const int nn = (int)G.nodes.size();
  std::vector<int> uses(nn, 0);
  for (const GNode& nd : G.nodes) {
    if (nd.a >= 0) ++uses[nd.a];
    if (nd.b >= 0) ++uses[nd.b];
    if (nd.c >= 0) ++uses[nd.c];
  }
  for (int k = 0; k < 8; ++k) uses[G.out[k]] += 2;
  std::vector<char> dead(nn, 0);
  for (int i = 0; i < nn; ++i) {
    GNode& nd = G.nodes[i];
    if (nd.op != G_AXPB || nd.pop || nd.a < 0 || uses[nd.a] != 1 || dead[nd.a]) continue;
    const GNode& s = G.nodes[nd.a];
    // exp takes an epilogue too (its transpose reads y - pt = ps exp), when it
    // has no folded sum.
    const bool ex = (s.op == G_EXP || s.op == G_STEXP) && !s.pop;
    if (!(generic_op(s.op) || ex) || s.ps != 1.0 || s.pt != 0.0) continue;
    GNode f = s;
    f.ps = nd.c0;
    f.pt = nd.c1;
    dead[nd.a] = 1;
    nd = f;
  }
  compact(G, dead);
}

// A sum or difference one of whose operands feeds nothing else becomes that
// operand's folded sum (c, pop): v + C, v - C or C - v.  The operand keeps its
// own op; its transpose takes +-1 times the cotangent and C's gradient the
// cotangent itself.  Exp and sqrt stay apart (their transposes read their own
// value), and so do the nodes with their own kernels or without a gradient,
// and C may not be an operand of the node it joins.
static bool generic_op(int op) {
  return op == G_STENCIL || op == G_STBIN || op == G_STMUL || op == G_ST2 || op == G_NB3 ||
         op == G_SHIFT ||
         op == G_ADD || op == G_SUB || op == G_MUL || op == G_DIV || op == G_MAX ||
         op == G_LOG || op == G_LOG1P || op == G_ABS || op == G_AXPB || op == G_CLAMPMIN ||
         op == G_CLAMPMAX;
}

static void fold_sums(GraphDef& G) {
  const int nn = (int)G.nodes.size();
  std::vector<int> uses(nn, 0);
  for (const GNode& nd : G.nodes) {
    if (nd.a >= 0) ++uses[nd.a];
    if (nd.b >= 0) ++uses[nd.b];
    if (nd.c >= 0) ++uses[nd.c];
  }
  for (int k = 0; k < 8; ++k) uses[G.out[k]] += 2;
  std::vector<char> dead(nn, 0);
  for (int i = 0; i < nn; ++i) {
    GNode& nd = G.nodes[i];
    if ((nd.op != G_ADD && nd.op != G_SUB) || nd.pop || nd.a == nd.b) continue;
    for (int side = 0; side < 2; ++side) {
      const int src = side == 0 ? nd.a : nd.b, oth = side == 0 ? nd.b : nd.a;
      if (src < 0 || oth < 0 || dead[src] || uses[src] != 1) continue;
      const GNode& s = G.nodes[src];
      if (!generic_op(s.op) || s.pop || s.ps != 1.0 || s.pt != 0.0) continue;
      if (s.a == oth || s.b == oth) continue;
      GNode f = s;
      f.c = oth;
      f.pop = nd.op == G_ADD ? 1 : (side == 0 ? 2 : 3);
      dead[src] = 1;
      nd = f;
      break;
    }
  }
  compact(G, dead);
}

// The 3-cell max and sum along an axis, built as (shift(a, s) op a) op
// shift(a, -s) from single-use shifts and an inner node of the same op (max or
// add), become one node (G_NB3) that reads the three neighbours itself.
static void fuse_neighbour3(GraphDef& G) {
  const int nn = (int)G.nodes.size();
  std::vector<int> uses(nn, 0);
  for (const GNode& nd : G.nodes) {
    if (nd.a >= 0) ++uses[nd.a];
    if (nd.b >= 0) ++uses[nd.b];
  }
  for (int k = 0; k < 8; ++k) uses[G.out[k]] += 2;
  std::vector<char> dead(nn, 0);
  auto lone = [&](int i, int op) {
    return i >= 0 && !dead[i] && uses[i] == 1 && G.nodes[i].op == op;
  };
  for (int i = 0; i < nn; ++i) {
    GNode& nd = G.nodes[i];
    if (nd.op != G_MAX && nd.op != G_ADD) continue;
    for (int side = 0; side < 2; ++side) {
      const int in = side == 0 ? nd.a : nd.b, s2 = side == 0 ? nd.b : nd.a;
      if (!lone(in, nd.op) || !lone(s2, G_SHIFT)) continue;
      const GNode& I = G.nodes[in];
      const GNode& S2 = G.nodes[s2];
      const int base = S2.a;
      const int s1 = I.a == base ? I.b : I.b == base ? I.a : -1;
      if (!lone(s1, G_SHIFT)) continue;
      const GNode& S1 = G.nodes[s1];
      if (S1.a != base || S1.axis != S2.axis || S1.sk != -S2.sk || (S1.sk != 1 && S1.sk != -1))
        continue;
      GNode f = nd;
      f.op = G_NB3;
      f.iop = nd.op;
      f.a = base;
      f.b = -1;
      f.axis = S1.axis;
      f.sk = S1.sk;
      f.c0 = f.c1 = 0;
      dead[in] = dead[s1] = dead[s2] = 1;
      nd = f;
      break;
    }
  }
  compact(G, dead);
}

void plan_reverse(const GraphDef& G, ReversePlan& P) {
  const int nn = (int)G.nodes.size();
  P.hasg.assign(nn, 0);
  P.wa.assign(nn, 0);
  P.wb.assign(nn, 0);
  P.wc.assign(nn, 0);
  P.gslot.assign(nn, -1);
  P.gprev.assign(nn, -1);
  P.nslots = 0;
  std::vector<int> freel, last_reader;   // free arrays; per array, its last reader
  auto take = [&](int x) {
    if (P.gslot[x] >= 0) return;
    if (!freel.empty()) {
      P.gslot[x] = freel.back();
      freel.pop_back();
      P.gprev[x] = last_reader[P.gslot[x]];
    } else {
      P.gslot[x] = P.nslots++;
      last_reader.push_back(-1);
    }
  };
  std::vector<char> seen(nn, 0);
  for (int k = 0; k < 8; ++k) {
    seen[G.out[k]] = P.hasg[G.out[k]] = 1;
    take(G.out[k]);   // the seeds
  }
  for (int i = nn - 1; i >= 0; --i) {
    const GNode& nd = G.nodes[i];
    if (!P.hasg[i] || !has_transpose(nd.op)) continue;
    if (nd.a >= 0) { P.wa[i] = !seen[nd.a]; seen[nd.a] = P.hasg[nd.a] = 1; take(nd.a); }
    if (nd.b >= 0) { P.wb[i] = !seen[nd.b]; seen[nd.b] = P.hasg[nd.b] = 1; take(nd.b); }
    if (nd.c >= 0) { P.wc[i] = !seen[nd.c]; seen[nd.c] = P.hasg[nd.c] = 1; take(nd.c); }
    // Node i's transpose has read its gradient: the array is free for the
    // nodes after it in the sweep (not an input's, read at the end).
    last_reader[P.gslot[i]] = i;
    freel.push_back(P.gslot[i]);
  }
}

// Drop the absorbed nodes and renumber every reference.
static void compact(GraphDef& G, const std::vector<char>& dead) {
  const int nn = (int)G.nodes.size();
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
    if (nd.c >= 0) nd.c = id[nd.c];
  }
  for (int k = 0; k < 8; ++k) {
    G.in[k] = id[G.in[k]];
    G.out[k] = id[G.out[k]];
  }
  G.nodes.swap(kept);
  G.memo.clear();
}

void build_rhs_graph(GraphDef& G, const stagger_grid& gr, const stagger_params& p, bool fuse) {
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
  if (fuse) {
    fuse_neighbour3(G);
    fuse_stencil_pairs(G);
    fold_sums(G);
    fold_affine(G);
  }
  for (GNode& nd : G.nodes) {
    nd.f0 = (float)nd.c0;
    nd.f1 = (float)nd.c1;
    nd.f2 = (float)nd.c2;
    nd.fh2 = (float)nd.h2;
    nd.fps = (float)nd.ps;
    nd.fpt = (float)nd.pt;
    nd.ep = nd.ps != 1.0 || nd.pt != 0.0;
  }
}

}  // namespace stg
