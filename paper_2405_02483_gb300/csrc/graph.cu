// Op-graph executor (see graph.cuh): one launch of a primitive's forward or
// transpose kernel (graph_kernels.cuh) per node, on one stream or as a DAG
// over several.
#include <math.h>

#include <stdint.h>

#include <algorithm>

#include "graph_kernels.cuh"

namespace stg {

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
      cudaMalloc(&qscr, sizeof(T) * 15 * (size_t)g.n) != cudaSuccess) {
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
  // Reverse-sweep bookkeeping: gradient flags and the reused gradient arrays.
  plan_reverse(def, rp);
  if (with_grads) {
    if (cudaMalloc(&grads, sizeof(T) * (size_t)rp.nslots * g.n) != cudaSuccess) {
      grads = nullptr;
      release();
      return STAGGER_EOOM;
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

// z extent of the launch: GBZ * GZU cells per block along z (GZU per thread).
static inline dim3 ggrid(const Geo& g) {
  return dim3((unsigned)((g.nx + GBX - 1) / GBX), (unsigned)((g.ny + GBY - 1) / GBY),
              (unsigned)((g.nz + GBZ * GZU - 1) / (GBZ * GZU)));
}

// The forward and transpose kernel of each op (the op a template constant):
// the stencil-like ops on the 3-D launch grid, the pointwise ops as flat
// kernels (pointwise_op).
template <typename T>
using FwdK = void (*)(GNode, const T*, const T*, const T*, T*, const T*, Geo);
template <typename T>
using BwdK = void (*)(GNode, const T*, const T*, const T*, const T*, T*, T*, T*, int, int, int,
                      Geo);
template <typename T>
using FwdPwK = void (*)(GNode, const T*, const T*, const T*, T*, long long, int);
template <typename T>
using BwdPwK = void (*)(GNode, const T*, const T*, const T*, const T*, T*, T*, T*, int, int, int,
                        long long, int);

template <typename T>
static FwdK<T> fwd_kernel(int op) {
  switch (op) {
    case G_STENCIL: return g_forward<T, G_STENCIL>;
    case G_SHIFT: return g_forward<T, G_SHIFT>;
    case G_STBIN: return g_forward<T, G_STBIN>;
    case G_STMUL: return g_forward<T, G_STMUL>;
    case G_ST2: return g_forward<T, G_ST2>;
    case G_STEXP: return g_forward<T, G_STEXP>;
    case G_NB3: return g_forward<T, G_NB3>;
    default: return g_forward<T, G_ZFIELD>;
  }
}

template <typename T>
static BwdK<T> bwd_kernel(int op) {
  switch (op) {
    case G_STENCIL: return g_backward<T, G_STENCIL>;
    case G_STBIN: return g_backward<T, G_STBIN>;
    case G_STMUL: return g_backward<T, G_STMUL>;
    case G_ST2: return g_backward<T, G_ST2>;
    case G_STEXP: return g_backward<T, G_STEXP>;
    case G_NB3: return g_backward<T, G_NB3>;
    default: return g_backward<T, G_SHIFT>;
  }
}

template <typename T>
static FwdK<T> fwd_kernel4(int op) {
  switch (op) {
    case G_STENCIL: return g_forward4<T, G_STENCIL>;
    case G_SHIFT: return g_forward4<T, G_SHIFT>;
    case G_STBIN: return g_forward4<T, G_STBIN>;
    case G_STMUL: return g_forward4<T, G_STMUL>;
    case G_ST2: return g_forward4<T, G_ST2>;
    case G_STEXP: return g_forward4<T, G_STEXP>;
    case G_NB3: return g_forward4<T, G_NB3>;
    default: return g_forward4<T, G_ZFIELD>;
  }
}

template <typename T>
static BwdK<T> bwd_kernel4(int op) {
  switch (op) {
    case G_STENCIL: return g_backward4<T, G_STENCIL>;
    case G_STBIN: return g_backward4<T, G_STBIN>;
    case G_STMUL: return g_backward4<T, G_STMUL>;
    case G_ST2: return g_backward4<T, G_ST2>;
    case G_STEXP: return g_backward4<T, G_STEXP>;
    case G_NB3: return g_backward4<T, G_NB3>;
    default: return g_backward4<T, G_SHIFT>;
  }
}

template <typename T>
static FwdPwK<T> fwd_kernel_pw(int op) {
  switch (op) {
    case G_ADD: return g_forward_pw<T, G_ADD>;
    case G_SUB: return g_forward_pw<T, G_SUB>;
    case G_MUL: return g_forward_pw<T, G_MUL>;
    case G_DIV: return g_forward_pw<T, G_DIV>;
    case G_MAX: return g_forward_pw<T, G_MAX>;
    case G_EXP: return g_forward_pw<T, G_EXP>;
    case G_LOG: return g_forward_pw<T, G_LOG>;
    case G_LOG1P: return g_forward_pw<T, G_LOG1P>;
    case G_SQRT: return g_forward_pw<T, G_SQRT>;
    case G_ABS: return g_forward_pw<T, G_ABS>;
    case G_AXPB: return g_forward_pw<T, G_AXPB>;
    case G_CLAMPMIN: return g_forward_pw<T, G_CLAMPMIN>;
    case G_CLAMPMAX: return g_forward_pw<T, G_CLAMPMAX>;
    case G_STEP: return g_forward_pw<T, G_STEP>;
    default: return g_forward_pw<T, G_CONST>;
  }
}

template <typename T>
static BwdPwK<T> bwd_kernel_pw(int op) {
  switch (op) {
    case G_ADD: return g_backward_pw<T, G_ADD>;
    case G_SUB: return g_backward_pw<T, G_SUB>;
    case G_MUL: return g_backward_pw<T, G_MUL>;
    case G_DIV: return g_backward_pw<T, G_DIV>;
    case G_MAX: return g_backward_pw<T, G_MAX>;
    case G_EXP: return g_backward_pw<T, G_EXP>;
    case G_LOG: return g_backward_pw<T, G_LOG>;
    case G_LOG1P: return g_backward_pw<T, G_LOG1P>;
    case G_SQRT: return g_backward_pw<T, G_SQRT>;
    case G_ABS: return g_backward_pw<T, G_ABS>;
    case G_AXPB: return g_backward_pw<T, G_AXPB>;
    case G_CLAMPMIN: return g_backward_pw<T, G_CLAMPMIN>;
    default: return g_backward_pw<T, G_CLAMPMAX>;
  }
}

// Flat launch of a pointwise kernel: four cells a thread when every array is
// 16-byte aligned and n a multiple of 4.
static inline bool al16(const void* p) { return ((uintptr_t)p & 15) == 0; }
// The four-x-cell stencil kernels: nx a multiple of 4 and shifts of one cell
// (the arrays' alignment is checked per launch), for the kernels they made
// faster.  The forward STMUL, which gathers two tap arrays, measured slower
// with four cells (FP32, 128^3, ncu launch list: 16.8 us at 64 registers
// against 15.9 with one cell) and keeps one cell a thread; every other
// forward (ST2 17.5 against 19.2 once its two stencils were formed one after
// the other) and every transpose is faster with four.
static inline bool cells4(const GNode& nd, const Geo& g, bool bwd) {
  if (g.nx % 4 != 0) return false;
  if ((nd.op == G_SHIFT || nd.op == G_NB3) && nd.sk != 1 && nd.sk != -1) return false;
  return bwd || nd.op != G_STMUL;
}
static inline dim3 ggrid4(const Geo& g) {
  return dim3((unsigned)((g.nx / 4 + GBX - 1) / GBX), (unsigned)((g.ny + GBY - 1) / GBY),
              (unsigned)((g.nz + GBZ - 1) / GBZ));
}
static inline unsigned pw_blocks(long long work) {
  const long long b = (work + 255) / 256;
  return (unsigned)(b < 8192 ? (b > 0 ? b : 1) : 8192);
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
    const T* C = nd.c >= 0 ? ptr[nd.c] : nullptr;
    cudaStream_t st = s;
    if (nconc) {
      // Follow the first operand's stream (chains stay on one stream); a node
      // without a computed operand starts the next stream in turn.
      int k = (nd.a >= 0 && sto[nd.a] >= 0) ? sto[nd.a]
            : (nd.b >= 0 && sto[nd.b] >= 0) ? sto[nd.b]
            : (nd.c >= 0 && sto[nd.c] >= 0) ? sto[nd.c] : (rr++ % nconc);
      st = aux[k];
      for (int o : {nd.a, nd.b, nd.c})
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
      if (geo.nx % 4 == 0 && al16(A) && al16(ptr[i]))
        g_quench_f4<T><<<ggrid4(geo), gb, 0, st>>>(nd, A, ptr[i], geo);
      else
        g_quench_f<T><<<gg, gb, 0, st>>>(nd, A, ptr[i], geo);
      ++launches;
    } else {
      if (pointwise_op(nd.op)) {
        const int vec = geo.n % 4 == 0 && al16(A) && al16(B) && al16(C) && al16(ptr[i]);
        fwd_kernel_pw<T>(nd.op)<<<pw_blocks(vec ? geo.n / 4 : geo.n), 256, 0, st>>>(
            nd, A, B, C, ptr[i], geo.n, vec);
      } else if (cells4(nd, geo, false) && al16(A) && al16(B) && al16(C) && al16(ptr[i])) {
        fwd_kernel4<T>(nd.op)<<<ggrid4(geo), gb, 0, st>>>(nd, A, B, C, ptr[i], mesh, geo);
      } else {
        fwd_kernel<T>(nd.op)<<<gg, gb, 0, st>>>(nd, A, B, C, ptr[i], mesh, geo);
      }
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
    STG_CUDA_OK(cudaMemcpyAsync(gptr(def.out[k]), seed[k],
                                sizeof(T) * geo.n, cudaMemcpyDeviceToDevice, s));
  // Concurrent form: the last launch that wrote each gradient array (-1: none
  // since the fork), and its stream.
  std::vector<int> lastw(nconc ? nn : 0, -1), sto(nconc ? nn : 0, -1);
  int rr = 0, prev_scr = -1;
  if (nconc && fork_streams(*this, s)) return STAGGER_ECUDA;
  const std::vector<char>&wa = rp.wa, &wb = rp.wb, &wc = rp.wc;
  for (long long i = (long long)nn - 1; i >= 0; --i) {
    const GNode& nd = def.nodes[i];
    if (!rp.hasg[i] || !has_transpose(nd.op)) continue;
    const T* A = nd.a >= 0 ? ptr[nd.a] : nullptr;
    const T* B = nd.b >= 0 ? ptr[nd.b] : nullptr;
    T* gA = nd.a >= 0 ? gptr(nd.a) : nullptr;
    T* gB = nd.b >= 0 ? gptr(nd.b) : nullptr;
    T* gC = nd.c >= 0 ? gptr(nd.c) : nullptr;
    cudaStream_t st = s;
    if (nconc) {
      // Wait for the complete gradient of this node, for the previous writer
      // of each gradient it adds to, for the transpose that last read an
      // array this launch writes first, and for the previous user of the
      // shared scratch (quench, plane mean).
      const int own = lastw[i];
      int k = own >= 0 ? sto[own] : (rr++ % nconc);
      st = aux[k];
      const bool scr = nd.op == G_QUENCH || nd.op == G_PMEAN;
      for (int w : {own, nd.a >= 0 ? lastw[nd.a] : -1, nd.b >= 0 ? lastw[nd.b] : -1,
                    nd.c >= 0 ? lastw[nd.c] : -1, scr ? prev_scr : -1,
                    wa[i] ? rp.gprev[nd.a] : -1, wb[i] ? rp.gprev[nd.b] : -1,
                    wc[i] ? rp.gprev[nd.c] : -1})
        if (w >= 0 && sto[w] != k) STG_CUDA_OK(cudaStreamWaitEvent(st, evn[w], 0));
      sto[i] = k;
      if (scr) prev_scr = (int)i;
    }
    if (nd.op == G_PMEAN) {
      g_plane_sum<T><<<geo.nz, 256, 0, st>>>(gptr((int)i), psum, geo);
      g_plane_bcast<T><<<gg, gb, 0, st>>>(psum, gA, wa[i] ? 0 : 1, geo);
      launches += 2;
    } else if (nd.op == G_QUENCH) {
      T* Q = qscr + (size_t)7 * geo.n;   // q and its derivatives, 4 arrays per axis slot
      T* gi = gptr((int)i);
      if (geo.nx % 4 == 0 && al16(A) && al16(gi) && al16(gA) && al16(qscr)) {
        const dim3 g4 = ggrid4(geo);
        g_quench_q4<T><<<g4, gb, 0, st>>>(nd, A, Q, geo);
        g_quench_b1_4<T><<<g4, gb, 0, st>>>(nd, A, Q, gi, qscr, geo);
        g_quench_b3_4<T><<<g4, gb, 0, st>>>(nd, Q, qscr, gA, wa[i], geo);
      } else {
        g_quench_q<T><<<gg, gb, 0, st>>>(nd, A, Q, geo);
        g_quench_b1<T><<<gg, gb, 0, st>>>(nd, A, Q, gi, qscr, geo);
        g_quench_b3<T><<<gg, gb, 0, st>>>(nd, Q, qscr, gA, wa[i], geo);
      }
      launches += 3;
    } else {
      T* gi = gptr((int)i);
      if (pointwise_op(nd.op)) {
        const int vec = geo.n % 4 == 0 && al16(A) && al16(B) && al16(ptr[i]) && al16(gi) &&
                        al16(gA) && al16(gB) && al16(gC);
        bwd_kernel_pw<T>(nd.op)<<<pw_blocks(vec ? geo.n / 4 : geo.n), 256, 0, st>>>(
            nd, A, B, ptr[i], gi, gA, gB, gC, wa[i], wb[i], wc[i], geo.n, vec);
      } else if (cells4(nd, geo, true) && al16(A) && al16(B) && al16(ptr[i]) && al16(gi) &&
                 al16(gA) && al16(gB) && al16(gC)) {
        bwd_kernel4<T>(nd.op)<<<ggrid4(geo), gb, 0, st>>>(nd, A, B, ptr[i], gi, gA, gB, gC,
                                                          wa[i], wb[i], wc[i], geo);
      } else {
        bwd_kernel<T>(nd.op)<<<gg, gb, 0, st>>>(nd, A, B, ptr[i], gi, gA, gB, gC, wa[i], wb[i],
                                                wc[i], geo);
      }
      ++launches;
    }
    if (nconc) {
      STG_CUDA_OK(cudaEventRecord(evn[i], st));
      if (nd.a >= 0) lastw[nd.a] = (int)i;
      if (nd.b >= 0) lastw[nd.b] = (int)i;
      if (nd.c >= 0) lastw[nd.c] = (int)i;
    }
  }
  if (nconc && join_streams(*this, s)) return STAGGER_ECUDA;
  Add8<T> ad;
  unsigned na = 0;
  int vec = geo.n % 4 == 0;
  for (int k = 0; k < 8; ++k) {
    if (!rp.hasg[def.in[k]]) continue;   // the outputs do not depend on this input
    ad.dst[na] = gin[k];
    ad.src[na] = gptr(def.in[k]);
    vec &= al16(ad.dst[na]) && al16(ad.src[na]);
    ++na;
  }
  if (na) {
    g_add_into8<T><<<dim3(pw_blocks(vec ? geo.n / 4 : geo.n), na), bs, 0, s>>>(ad, geo.n, vec);
    ++launches;
  }
  STG_CUDA_OK(cudaGetLastError());
  return STAGGER_OK;
}

template struct GraphExec<float>;
template struct GraphExec<double>;

}  // namespace stg
