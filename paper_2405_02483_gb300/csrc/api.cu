// C ABI of libstagger (declared in include/stagger.h).
#include <math.h>
#include <string.h>

#include <stdint.h>

#include <algorithm>
#include <new>

#include "fused.cuh"
#include "graph_kernels.cuh"

using namespace stg;

struct stagger_ctx {
  stagger_grid grid;
  stagger_params params;
  Geo geo;
  Fused fused;
  GraphDef gdef;
  GraphExec<float>* g32 = nullptr;
  GraphExec<double>* g64 = nullptr;
  float* w32 = nullptr;    // adjoint workspace: f1, f2, q, fbar, qbar (8 each)
  double* w64 = nullptr;
  float* host_state = nullptr;  // device copy for stagger_step_host
  long long extra_launches = 0;
  // The adjoint step as a captured CUDA graph per precision (0 FP32, 1 FP64):
  // state 0 not tried, 1 captured, -1 capture unavailable (direct launches).
  int adj_state[2] = {0, 0};
  cudaGraphExec_t adj_exec[2] = {nullptr, nullptr};
  long long adj_launches[2] = {0, 0};
  cudaStream_t cap = nullptr;
  double* dtp = nullptr;   // the step dt on the device (read by the captured graph),
                           // then beta_s dt of the three RK stages
  float* bdtf = nullptr;   // beta_s dt in FP32
  double* omean_g = nullptr;  // plane means and parts of the op graph's open boundaries
};

namespace stg {

// Argument checks shared by stagger_create and stagger_diagnostics_noalloc.
int validate_inputs(const stagger_grid* g, const stagger_params* p) {
  if (!g || !p) return STAGGER_EINVAL;
  if (g->nx < 1 || g->ny < 1 || g->nz < 1) return STAGGER_EINVAL;
  if (!(g->dx > 0) || !(g->dy > 0) || !(g->dz > 0)) return STAGGER_EINVAL;
  long long n = (long long)g->nx * g->ny * g->nz;
  if (n >= (1LL << 31)) return STAGGER_EINVAL;  // 32-bit cell offsets in the kernels
  // Launch grids put y and z (over 1 to 8 cells a block) on the 65535-block axes.
  if (g->ny > 65535 || g->nz > 65535) return STAGGER_EINVAL;
  if (!(p->gamma > 1.0)) return STAGGER_EINVAL;
  if (p->nu1 < 0 || p->nu2 < 0 || p->nu3 < 0 || p->nu_const < 0 || p->nuE < 0 || p->nuB < 0 ||
      p->csmag < 0)
    return STAGGER_EINVAL;
  if (p->do_quench && (!(p->qmax > 0) || !(p->qlim > 0))) return STAGGER_EINVAL;
  if (!(p->Cdt > 0) || !(p->Cdtr > 0) || !(p->Cdtd > 0)) return STAGGER_EINVAL;
  if (p->ref[0] < 0) return STAGGER_EINVAL;
  if (!(p->t_cool >= 0) || !isfinite(p->e_cool)) return STAGGER_EINVAL;
  if (p->cool_cut < 0 || p->cool_cut > 2 || (p->cool_cut && !(p->rho_cool > 0))) return STAGGER_EINVAL;
  if (p->scalar_cells < 0 || p->scalar_cells > 1) return STAGGER_EINVAL;
  if (p->fuse_flux_div < 0 || p->fuse_flux_div > 1) return STAGGER_EINVAL;
  if (p->quench_max3 < 0 || p->quench_max3 > 1 || !(p->quench_eps >= 0) || !isfinite(p->quench_eps))
    return STAGGER_EINVAL;
  if (p->zwalls < 0 || p->zwalls > 3) return STAGGER_EINVAL;
  if (!(p->top_tpot >= 0) || !isfinite(p->top_tpot)) return STAGGER_EINVAL;
  // The potential-field transforms keep nx complex roots in shared memory.
  if (p->zwalls == 3 && p->top_tpot > 0 && g->nx > 24576) return STAGGER_EINVAL;
  if (p->zwalls == 3) {   // stellar-atmosphere boundaries
    const double v[] = {p->bdry_t, p->bdry_rho, p->bdry_E, p->bdry_u, p->bdry_B[0],
                        p->bdry_B[1], p->bdry_B[2], p->top_rho_lo, p->top_rho_hi,
                        p->top_e_fac, p->top_umax, p->top_tpot};
    for (double x : v)
      if (!isfinite(x)) return STAGGER_EINVAL;
    if (!(p->bdry_t > 0) || !(p->bdry_rho > 0) || !(p->bdry_E > 0) || !(p->bdry_u > 0) ||
        !(p->top_umax > 0) || !(p->top_tpot >= 0) || !(p->top_rho_lo > 0) || p->top_rho_lo > 1 ||
        p->top_rho_hi < 1 || p->top_e_fac < 1 || p->g[2] == 0 || p->fuse_flux_div ||
        g->nz < 3 * p->zghost + 2)
      return STAGGER_EINVAL;
  }
  if (p->ediffav < 0 || p->ediffav > 1) return STAGGER_EINVAL;
  if (p->lnp_aver < 0 || p->lnp_aver > 1) return STAGGER_EINVAL;
  if (p->lnp_aver && p->fuse_flux_div) return STAGGER_EINVAL;
  // z walls (closed or rigid): at least the reach of the right-hand side in ghost planes
  // at each end, one physical spacing between the boundary planes, uniform z.
  if (p->zwalls && (p->zghost < STAGGER_ZGHOST_MIN || g->nz < 2 * p->zghost + 2 || p->zc ||
                    p->csmag > 0))
    return STAGGER_EINVAL;
  // The reflection acts on the stored deviations: the odd fields need a zero background.
  if (p->zwalls == 1 && (p->ref[3] != 0 || p->ref[5] != 0 || p->ref[6] != 0))
    return STAGGER_EINVAL;
  if (p->do_2nddiv < 0 || p->do_2nddiv > 1 || !isfinite(p->d2lnr_lim)) return STAGGER_EINVAL;
  for (int k = 0; k < 8; ++k)
    if (!isfinite(p->ref[k])) return STAGGER_EINVAL;
  if (!(p->t_chromo >= 0) || (p->t_chromo > 0 && !(p->rho_bot > 0))) return STAGGER_EINVAL;
  if (!(p->cor_L0 >= 0) || (p->cor_L0 > 0 && !(p->cor_Tunit > 0))) return STAGGER_EINVAL;
  if (!isfinite(p->t_chromo) || !isfinite(p->cor_L0) || !isfinite(p->rho_bot) ||
      !isfinite(p->cor_Tunit))
    return STAGGER_EINVAL;
  if ((p->zc == nullptr) != (p->zf == nullptr)) return STAGGER_EINVAL;
  if (p->zc) {
    if (g->nz < 2) return STAGGER_EINVAL;
    for (int k = 0; k < g->nz; ++k)
      if (!(p->zc[k] > 0) || !(p->zf[k] > 0) || !isfinite(p->zc[k]) || !isfinite(p->zf[k]))
        return STAGGER_EINVAL;
  }
  return STAGGER_OK;
}

}  // namespace stg

extern "C" {

int stagger_params_default(stagger_params* p) {
  if (!p) return STAGGER_EINVAL;
  memset(p, 0, sizeof(*p));
  p->gamma = 5.0 / 3.0;
  p->nuE = 1.0;
  p->nuB = 1.0;
  p->qmax = 8.0;
  p->qlim = 2.0;
  p->quench_eps = 1e-4;
  p->log_interp = 1;
  p->Cdt = 0.4;
  p->Cdtr = 0.1;
  p->Cdtd = 0.7;
  p->rho_cool = 1.0;
  p->d2lnr_lim = 0.3;
  p->rho_bot = 1.0;
  p->cor_Tunit = 1.0;
  p->bdry_t = p->bdry_rho = p->bdry_E = p->bdry_u = 1.0;
  p->top_rho_lo = 0.5;
  p->top_rho_hi = 2.0;
  p->top_e_fac = 2.0;
  p->top_umax = 1.0;
  return STAGGER_OK;
}

const char* stagger_strerror(int s) {
  switch (s) {
    case STAGGER_OK: return "ok";
    case STAGGER_EINVAL: return "invalid argument";
    case STAGGER_ECUDA: return "CUDA runtime error";
    case STAGGER_ENONFINITE: return "non-finite value in the state";
    case STAGGER_EOOM: return "device memory allocation failed";
    case STAGGER_ETIMEOUT: return "bounded device wait timed out";
    case STAGGER_EUNSUPPORTED: return "unsupported feature";
    default: return "unknown status";
  }
}

int stagger_create(const stagger_grid* grid, const stagger_params* params, stagger_ctx** out) {
  if (!out) return STAGGER_EINVAL;
  *out = nullptr;
  int rc = validate_inputs(grid, params);
  if (rc) return rc;
  stagger_ctx* c = new (std::nothrow) stagger_ctx();
  if (!c) return STAGGER_EOOM;
  c->grid = *grid;
  c->params = *params;
  c->geo = make_geo(grid->nx, grid->ny, grid->nz);
  rc = fused_init(c->fused, *grid, *params);
  if (rc) {
    delete c;
    return rc;
  }
  build_rhs_graph(c->gdef, *grid, *params);
  // The mesh arrays are the caller's and were read above (the fused path and
  // the graph keep their own copies): drop the pointers.
  c->params.zc = c->params.zf = nullptr;
  *out = c;
  return STAGGER_OK;
}

int stagger_destroy(stagger_ctx* c) {
  if (!c) return STAGGER_OK;
  cudaError_t e = cudaDeviceSynchronize();
  fused_release(c->fused);
  if (c->g32) { c->g32->release(); delete c->g32; }
  if (c->g64) { c->g64->release(); delete c->g64; }
  if (c->w32) cudaFree(c->w32);
  if (c->w64) cudaFree(c->w64);
  if (c->host_state) cudaFree(c->host_state);
  for (int i = 0; i < 2; ++i)
    if (c->adj_exec[i]) cudaGraphExecDestroy(c->adj_exec[i]);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->dtp) cudaFree(c->dtp);
  if (c->bdtf) cudaFree(c->bdtf);
  if (c->omean_g) cudaFree(c->omean_g);
  delete c;
  return e == cudaSuccess ? STAGGER_OK : STAGGER_ECUDA;
}

size_t stagger_cells(const stagger_ctx* c) { return c ? (size_t)c->geo.n : 0; }

long long stagger_launch_count(const stagger_ctx* c) {
  if (!c) return 0;
  long long n = c->fused.launches + c->extra_launches;
  if (c->g32) n += c->g32->launches;
  if (c->g64) n += c->g64->launches;
  return n;
}

static bool ptrs_ok(void* const* a) {
  if (!a) return false;
  for (int k = 0; k < 8; ++k)
    if (!a[k]) return false;
  return true;
}

int stagger_rhs(stagger_ctx* c, float* const state[8], float* dfdt[8], void* stream) {
  if (!c || !ptrs_ok((void* const*)state) || !ptrs_ok((void* const*)dfdt)) return STAGGER_EINVAL;
  return fused_rhs(c->fused, state, dfdt, (cudaStream_t)stream);
}

int stagger_step(stagger_ctx* c, float* state[8], double dt, double* dt_used, void* stream) {
  if (!c || !ptrs_ok((void* const*)state) || !(dt == dt)) return STAGGER_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = fused_step_graphed(c->fused, state, dt, s);
  if (rc) return rc;
  if (dt_used) {
    double h;
    STG_CUDA_OK(cudaMemcpyAsync(&h, c->fused.dt_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    STG_CUDA_OK(cudaStreamSynchronize(s));
    *dt_used = h;
  }
  return STAGGER_OK;
}

int stagger_run(stagger_ctx* c, float* state[8], int nsteps, double dt, void* stream) {
  if (!c || !ptrs_ok((void* const*)state) || nsteps < 0 || !(dt == dt)) return STAGGER_EINVAL;
  for (int i = 0; i < nsteps; ++i) {
    int rc = fused_step_graphed(c->fused, state, dt, (cudaStream_t)stream);
    if (rc) return rc;
  }
  return STAGGER_OK;
}

int stagger_timing(stagger_ctx* c, int on) {
  if (!c) return STAGGER_EINVAL;
  if (on && !c->fused.timing)
    for (int i = 0; i < K_COUNT; ++i) { c->fused.kt_ms[i] = 0; c->fused.kt_n[i] = 0; }
  fused_timing(c->fused, on ? 1 : 0);
  return STAGGER_OK;
}

int stagger_kernel_times(stagger_ctx* c, int max, const char** names, double* total_ms,
                         long long* launches, void* stream) {
  if (!c || max < 0) return STAGGER_EINVAL;
  int rc = fused_collect(c->fused, (cudaStream_t)stream);
  if (rc) return rc;
  for (int i = 0; i < K_COUNT && i < max; ++i) {
    if (names) names[i] = KNAMES[i];
    if (total_ms) total_ms[i] = c->fused.kt_ms[i];
    if (launches) launches[i] = c->fused.kt_n[i];
  }
  return K_COUNT;
}

int stagger_courant(stagger_ctx* c, float* const state[8], double* dt_host, double limits[3],
                    void* stream) {
  if (!c || !ptrs_ok((void* const*)state) || !dt_host) return STAGGER_EINVAL;
  return fused_courant(c->fused, state, limits, dt_host, (cudaStream_t)stream);
}

int stagger_dt(stagger_ctx* c, float* const state[8], double* out, int on_device, void* stream) {
  if (!c || !ptrs_ok((void* const*)state) || !out || on_device < 0 || on_device > 1)
    return STAGGER_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = fused_dt(c->fused, state, s);
  if (rc) return rc;
  if (on_device) {
    // Stream-ordered: copied before any later call on this stream rewrites it.
    STG_CUDA_OK(cudaMemcpyAsync(out, c->fused.dt_dev, 4 * sizeof(double),
                                cudaMemcpyDeviceToDevice, s));
    return STAGGER_OK;
  }
  double h[4];
  STG_CUDA_OK(cudaMemcpyAsync(h, c->fused.dt_dev, sizeof(h), cudaMemcpyDeviceToHost, s));
  STG_CUDA_OK(cudaStreamSynchronize(s));
  for (int i = 0; i < 4; ++i) out[i] = h[i];
  if (!(h[0] == h[0]) || h[0] <= 0) return STAGGER_ENONFINITE;
  return STAGGER_OK;
}

int stagger_diagnostics(stagger_ctx* c, float* const state[8], double out[10], void* stream) {
  if (!c || !ptrs_ok((void* const*)state) || !out) return STAGGER_EINVAL;
  return fused_diagnostics(c->fused, state, c->params, out, (cudaStream_t)stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Unfused graph path and the adjoint step.
// ---------------------------------------------------------------------------
// The scalars come in the sweep's precision (a conversion from double, or a
// double product, runs on the narrow FP64 pipe: not once per thread).
template <typename T>
__global__ void k_lin2(T* o, const T* x, T a, const T* y, T b, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = a * x[i] + b * y[i];
}
// o_k = a x_k + b_k y_k for the eight fields in one launch (blockIdx.y = k),
// b_k = *bdt when bdt is given (beta_s dt on the device), else b; four
// elements a thread through 16-byte accesses when vec.
template <typename T>
struct Lin8 {
  T* o[8];
  const T* x[8];
  const T* y[8];
};
template <typename T>
__global__ void k_lin2x8(Lin8<T> p, T a, T b, const T* bdt, long long n, int vec) {
  const int f = blockIdx.y;
  const T bb = bdt ? bdt[0] : b;
  T* o = p.o[f];
  const T *x = p.x[f], *y = p.y[f];
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (vec) {
    for (; t < n / 4; t += stride) {
      T xv[4], yv[4], ov[4];
      ld4(x, 4 * t, xv);
      ld4(y, 4 * t, yv);
#pragma unroll
      for (int l = 0; l < 4; ++l) ov[l] = a * xv[l] + bb * yv[l];
      st4(o, 4 * t, ov);
    }
  } else {
    for (; t < n; t += stride) o[t] = a * x[t] + bb * y[t];
  }
}

// dt, and beta_s dt of the three RK stages in FP64 and FP32.
__global__ void k_set_dt3(double* dtp, float* bdtf, double dt, double b0, double b1, double b2) {
  const double b[3] = {b0, b1, b2};
  dtp[0] = dt;
  for (int s = 0; s < 3; ++s) {
    dtp[1 + s] = b[s] * dt;
    bdtf[s] = (float)(b[s] * dt);
  }
}
template <typename T>
__global__ void k_copy(T* o, const T* x, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = x[i];
}

// Rigid z walls (reading R25) around the op graph: the ghost momenta of a
// state from its boundary planes' velocity, p_d(k) = rho_d(k) u_d(b), rho_d
// formed as the graph forms it (eq. (interp) on ln(rho/r0), or on rho without
// log interpolation), and the ghost planes of a derivative zeroed.  Planes
// outside lb..ub are ghost planes for every field.
template <typename T>
struct RigidG {
  T* p[3];
  const T* rd;
  double r0, pref[3];
  int log_interp;
};
template <typename T>
__global__ void k_rigid_fill_g(RigidG<T> a, int lb, int ub, Geo g) {
  const int d = blockIdx.z;
  const int pl = blockIdx.y;                   // planes 0..lb-1, then ub+1..nz-1
  const int kz = pl < lb ? pl : ub + 1 + (pl - lb);
  const long long m2 = (long long)g.nx * g.ny;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m2 || kz >= g.nz) return;
  const int ix = (int)(i % g.nx), jy = (int)(i / g.nx);
  const int b = kz < lb ? lb : ub;
  auto rho_face = [&](int z) {
    auto ls = [&](int o) {
      const double r = (double)a.rd[lin(g, wrap(ix + (d == 0 ? o : 0), g.nx),
                                        wrap(jy + (d == 1 ? o : 0), g.ny),
                                        wrap(z + (d == 2 ? o : 0), g.nz))];
      if (!a.log_interp) return r;
      return a.r0 > 0 ? log1p(r / a.r0) : log(r + a.r0);
    };
    // eq. (interp) to the lower face: weights 75/128, -25/256, 3/256
    const double v = (75.0 / 128.0) * (ls(-1) + ls(0)) + (-25.0 / 256.0) * (ls(-2) + ls(1)) +
                     (3.0 / 256.0) * (ls(-3) + ls(2));
    if (!a.log_interp) return v + a.r0;
    return a.r0 > 0 ? a.r0 * exp(v) : exp(v);
  };
  T* p = a.p[d];
  const double u = ((double)p[lin(g, ix, jy, b)] + a.pref[d]) / rho_face(b);
  p[lin(g, ix, jy, kz)] = (T)(rho_face(kz) * u - a.pref[d]);
}
template <typename T>
__global__ void k_zero_ghost_planes(T* o, int lb, int ub, Geo g) {
  const int pl = blockIdx.y;
  const int kz = pl < lb ? pl : ub + 1 + (pl - lb);
  const long long m2 = (long long)g.nx * g.ny;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m2 || kz >= g.nz) return;
  o[(long long)kz * m2 + i] = T(0);
}

template <typename T>
static void rigid_fill_g(stagger_ctx* c, T* const f[8], cudaStream_t s) {
  const stagger_params& p = c->params;
  const Geo& g = c->geo;
  const int lb = p.zghost, ub = g.nz - 1 - p.zghost;
  RigidG<T> a;
  for (int d = 0; d < 3; ++d) {
    a.p[d] = f[1 + d];
    a.pref[d] = p.ref[1 + d];
  }
  a.rd = f[0];
  a.r0 = p.ref[0];
  a.log_interp = p.log_interp;
  const dim3 gr((unsigned)((g.sz + 255) / 256), (unsigned)(lb + (g.nz - 1 - ub)), 3);
  k_rigid_fill_g<T><<<gr, 256, 0, s>>>(a, lb, ub, g);
  ++c->extra_launches;
}
template <typename T>
static void rigid_zero_g(stagger_ctx* c, T* o, cudaStream_t s) {
  const Geo& g = c->geo;
  const int lb = c->params.zghost, ub = g.nz - 1 - c->params.zghost;
  const dim3 gr((unsigned)((g.sz + 255) / 256), (unsigned)(lb + (g.nz - 1 - ub)));
  k_zero_ghost_planes<T><<<gr, 256, 0, s>>>(o, lb, ub, g);
  ++c->extra_launches;
}

// Stellar-atmosphere z boundaries (reading R26) around the op graph: the same
// ghost fill and boundary-plane rates as the fused path, in the graph's
// precision (see stagger_params.zwalls).
template <typename T>
struct OpenG {
  T* f[8];                       // the state (deviations)
  double ref[8];
  int lb, ub, bot, top, sb, st, log_interp;
  double inv_t, rho_b, E_b, inv_u, Bb[2], rlo, rhi, efac, umax, gabs, gamma, gm1, ihz;
  const double* mean;            // G top-ghost densities, then the p_x, p_y plane means
};
template <typename T>
__device__ double open_rho_face(const OpenG<T>& a, const Geo& g, int d, int ix, int jy, int z) {
  auto ls = [&](int o) {
    const double r = (double)a.f[0][lin(g, wrap(ix + (d == 0 ? o : 0), g.nx),
                                       wrap(jy + (d == 1 ? o : 0), g.ny),
                                       wrap(z + (d == 2 ? o : 0), g.nz))];
    if (!a.log_interp) return r;
    return a.ref[0] > 0 ? log1p(r / a.ref[0]) : log(r + a.ref[0]);
  };
  const double v = (75.0 / 128.0) * (ls(-1) + ls(0)) + (-25.0 / 256.0) * (ls(-2) + ls(1)) +
                   (3.0 / 256.0) * (ls(-3) + ls(2));
  if (!a.log_interp) return v + a.ref[0];
  return a.ref[0] > 0 ? a.ref[0] * exp(v) : exp(v);
}
template <typename T>
__global__ void k_open_part_g(OpenG<T> a, double* part, Geo g) {
  __shared__ double sm[256];
  const int row = blockIdx.y, nb = gridDim.x, G = a.lb;
  const long long m = (long long)g.nx * g.ny;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (long long)nb * blockDim.x) {
    if (row < G) {
      const double lb_ = log((double)a.f[0][(long long)a.top * m + i] + a.ref[0]);
      const double li = log((double)a.f[0][(long long)(a.top - a.st) * m + i] + a.ref[0]);
      acc += exp(lb_ + (row + 1) * (lb_ - li));
    } else {
      acc += (double)a.f[row == G ? 1 : 2][(long long)a.bot * m + i];
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
__global__ void k_open_final_g(const double* part, int nb, int rows, double* mean, Geo g) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(long long)r * nb + b];
  mean[r] = s / ((double)g.nx * g.ny);
}
// rho and E of the ghost centre planes (0..lb-1, then ub+1..nz-1).
template <typename T>
__global__ void k_open_fill_c_g(OpenG<T> a, Geo g) {
  const int lb = a.lb, ub = a.ub, pl = blockIdx.y;
  const int kz = pl < lb ? pl : ub + 1 + (pl - lb);
  const long long m2 = (long long)g.nx * g.ny;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m2 || kz >= g.nz) return;
  const bool low = kz < lb;
  const int b = low ? lb : ub, s = low ? -1 : 1, j = low ? lb - kz : kz - ub;
  T* rd = a.f[0];
  T* Ed = a.f[4];
  const double rb = (double)rd[(long long)b * m2 + i] + a.ref[0];
  const double ri = (double)rd[(long long)(b - s) * m2 + i] + a.ref[0];
  const double eb = ((double)Ed[(long long)b * m2 + i] + a.ref[4]) / rb;
  const double ei = ((double)Ed[(long long)(b - s) * m2 + i] + a.ref[4]) / ri;
  const double lrb = log(rb);
  double r = exp(lrb + j * (lrb - log(ri)));
  double e = eb + j * (eb - ei);
  if (b == a.top) {
    const double mj = a.mean[j - 1];
    r = fmin(fmax(r, a.rlo * mj), a.rhi * mj);
    e = fmin(fmax(e, eb / a.efac), eb * a.efac);
  }
  rd[(long long)kz * m2 + i] = (T)(r - a.ref[0]);
  Ed[(long long)kz * m2 + i] = (T)(r * e - a.ref[4]);
}
// Momenta and field of the ghost planes (0..lb, then ub+1..nz-1).
template <typename T>
__global__ void k_open_fill_m_g(OpenG<T> a, Geo g) {
  const int lb = a.lb, ub = a.ub, pl = blockIdx.y;
  const int kz = pl <= lb ? pl : ub + 1 + (pl - lb - 1);
  const long long m2 = (long long)g.nx * g.ny;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m2 || kz >= g.nz) return;
  const int ix = (int)(i % g.nx), jy = (int)(i / g.nx);
  const bool low = kz <= lb;
  const int b = low ? lb : ub, s = low ? -1 : 1, mi = low ? lb + 1 : ub;
  const bool centre = low ? kz < lb : true;
  const int j = low ? lb - kz : kz - ub;
  const bool top = b == a.top;
  auto at = [&](int z) { return (long long)z * m2 + i; };
  T *px = a.f[1], *py = a.f[2], *pz = a.f[3], *bx = a.f[5], *by = a.f[6], *bz = a.f[7];
  const double uzi = ((double)pz[at(mi)] + a.ref[3]) / open_rho_face(a, g, 2, ix, jy, mi);
  if (!top) {
    if (centre) {
      px[at(kz)] = px[at(2 * b - kz)];
      py[at(kz)] = py[at(2 * b - kz)];
    }
    pz[at(kz)] = pz[at(2 * b + 1 - kz)];
  } else {
    const double um = a.umax;
    if (centre) {
      const double ux = fmin(fmax(((double)px[at(b)] + a.ref[1]) / open_rho_face(a, g, 0, ix, jy, b), -um), um);
      const double uy = fmin(fmax(((double)py[at(b)] + a.ref[2]) / open_rho_face(a, g, 1, ix, jy, b), -um), um);
      px[at(kz)] = (T)(open_rho_face(a, g, 0, ix, jy, kz) * ux - a.ref[1]);
      py[at(kz)] = (T)(open_rho_face(a, g, 1, ix, jy, kz) * uy - a.ref[2]);
    }
    const double uz = fmin(fmax(uzi, -um), um);
    pz[at(kz)] = (T)(open_rho_face(a, g, 2, ix, jy, kz) * uz - a.ref[3]);
  }
  const int d = low ? mi - kz : kz - mi;
  bz[at(kz)] = (T)((double)bz[at(mi)] + d * ((double)bz[at(mi)] - (double)bz[at(mi - s)]));
  if (centre) {
    double vx = (double)bx[at(b)] + j * ((double)bx[at(b)] - (double)bx[at(b - s)]);
    double vy = (double)by[at(b)] + j * ((double)by[at(b)] - (double)by[at(b - s)]);
    if (!top) {
      const double f = 1.0 / (1.0 + exp(s * uzi * a.inv_u));
      vx = (1.0 - f) * vx + f * (a.Bb[0] - a.ref[5]);
      vy = (1.0 - f) * vy + f * (a.Bb[1] - a.ref[6]);
    }
    bx[at(kz)] = (T)vx;
    by[at(kz)] = (T)vy;
  }
}
// The boundary-plane rates on the graph's derivatives F (state filled), and
// zero derivatives on the ghost planes (centres outside lb..ub, z faces
// outside lb+1..ub).
template <typename T>
__global__ void k_open_rates_g(OpenG<T> a, T* F0, T* F1, T* F2, T* F4, Geo g) {
  const long long m2 = (long long)g.nx * g.ny;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m2) return;
  const int ix = (int)(i % g.nx), jy = (int)(i / g.nx);
  auto at = [&](int z) { return (long long)z * m2 + i; };
  const T *rd = a.f[0], *Ed = a.f[4], *pz = a.f[3];
  {  // bottom, eqs. (rein), (constS) to (addderiv)
    const int b = a.bot, mi = a.sb < 0 ? b + 1 : b;
    const double r = (double)rd[at(b)] + a.ref[0], E = (double)Ed[at(b)] + a.ref[4];
    const double ui = ((double)pz[at(mi)] + a.ref[3]) / open_rho_face(a, g, 2, ix, jy, mi);
    const double f = 1.0 / (1.0 + exp(a.sb * ui * a.inv_u));
    const double dE = (a.E_b - E) * a.inv_t;
    const double Fm = (double)F0[at(b)], Fe = (double)F4[at(b)];
    F0[at(b)] = (T)(f * (a.rho_b - r) * a.inv_t + (1.0 - f) * (Fm + (dE - Fe) * r / (a.gamma * E)));
    F4[at(b)] = (T)dE;
    F1[at(b)] = (T)((double)F1[at(b)] - f * ((double)a.f[1][at(b)] - a.mean[a.lb]) * a.inv_t);
    F2[at(b)] = (T)((double)F2[at(b)] - f * ((double)a.f[2][at(b)] - a.mean[a.lb + 1]) * a.inv_t);
  }
  {  // top, eq. (rbdrylo)
    const int t = a.top;
    const double r = (double)rd[at(t)] + a.ref[0], E = (double)Ed[at(t)] + a.ref[4];
    const double HP = a.gm1 * (E / r) / a.gabs;
    auto p = [&](int o) { return (double)pz[lin(g, ix, jy, wrap(t + o, g.nz))] + a.ref[3]; };
    const double du = ((225.0 / 192.0) * (p(1) - p(0)) + (-25.0 / 384.0) * (p(2) - p(-1)) +
                       (3.0 / 640.0) * (p(3) - p(-2))) * a.ihz;
    const double upz = (75.0 / 128.0) * (p(0) + p(1)) + (-25.0 / 256.0) * (p(-1) + p(2)) +
                       (3.0 / 256.0) * (p(-2) + p(3));
    F0[at(t)] = (T)((double)F0[at(t)] + du + a.st * upz / HP);
  }
}
template <typename T>
__global__ void k_open_zero_g(T* o, int face, int lb, int ub, Geo g) {
  const int pl = blockIdx.y;                   // planes 0..lb, then ub+1..nz-1
  const int kz = pl <= lb ? pl : ub + 1 + (pl - lb - 1);
  const long long m2 = (long long)g.nx * g.ny;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m2 || kz >= g.nz) return;
  if (kz == lb && !face) return;               // the centre plane lb is physical
  o[(long long)kz * m2 + i] = T(0);
}

template <typename T>
static OpenG<T> open_args(stagger_ctx* c, T* const f[8]) {
  const stagger_params& p = c->params;
  const Geo& g = c->geo;
  OpenG<T> a;
  for (int k = 0; k < 8; ++k) {
    a.f[k] = f[k];
    a.ref[k] = p.ref[k];
  }
  a.lb = p.zghost;
  a.ub = g.nz - 1 - p.zghost;
  a.bot = p.g[2] < 0 ? a.lb : a.ub;
  a.top = p.g[2] < 0 ? a.ub : a.lb;
  a.sb = p.g[2] < 0 ? -1 : 1;
  a.st = -a.sb;
  a.log_interp = p.log_interp;
  a.inv_t = 1.0 / p.bdry_t;
  a.rho_b = p.bdry_rho;
  a.E_b = p.bdry_E;
  a.inv_u = 1.0 / p.bdry_u;
  a.Bb[0] = p.bdry_B[0];
  a.Bb[1] = p.bdry_B[1];
  a.rlo = p.top_rho_lo;
  a.rhi = p.top_rho_hi;
  a.efac = p.top_e_fac;
  a.umax = p.top_umax;
  a.gabs = fabs(p.g[2]);
  a.gamma = p.gamma;
  a.gm1 = p.gamma - 1.0;
  a.ihz = 1.0 / c->grid.dz;
  a.mean = c->omean_g;
  return a;
}
template <typename T>
static int open_fill_g(stagger_ctx* c, T* const f[8], cudaStream_t s) {
  const Geo& g = c->geo;
  const int G = c->params.zghost, rows = G + 2;
  const int nb = (int)std::max(1LL, std::min(64LL, ((long long)g.nx * g.ny + 1023) / 1024));
  if (!c->omean_g &&
      cudaMalloc(&c->omean_g, sizeof(double) * (size_t)rows * (1 + nb)) != cudaSuccess) {
    c->omean_g = nullptr;
    return STAGGER_EOOM;
  }
  OpenG<T> a = open_args<T>(c, f);
  const unsigned bx = (unsigned)((g.sz + 255) / 256);
  k_open_part_g<T><<<dim3(nb, rows), 256, 0, s>>>(a, c->omean_g + rows, g);
  k_open_final_g<<<(rows + 63) / 64, 64, 0, s>>>(c->omean_g + rows, nb, rows, c->omean_g, g);
  k_open_fill_c_g<T><<<dim3(bx, 2 * G), 256, 0, s>>>(a, g);
  k_open_fill_m_g<T><<<dim3(bx, 2 * G + 1), 256, 0, s>>>(a, g);
  c->extra_launches += 4;
  STG_CUDA_OK(cudaGetLastError());
  return STAGGER_OK;
}
// After the graph's forward on the filled state f: the boundary-plane rates
// on its outputs and zero ghost derivatives.
template <typename T>
static void open_rates_g(stagger_ctx* c, T* const f[8], T* const F[8], cudaStream_t s) {
  const Geo& g = c->geo;
  OpenG<T> a = open_args<T>(c, f);
  k_open_rates_g<T><<<(unsigned)((g.sz + 255) / 256), 256, 0, s>>>(a, F[0], F[1], F[2], F[4], g);
  const dim3 gr((unsigned)((g.sz + 255) / 256), (unsigned)(2 * c->params.zghost + 1));
  for (int k = 0; k < 8; ++k)
    k_open_zero_g<T><<<gr, 256, 0, s>>>(F[k], k == 3 || k == 7, a.lb, a.ub, g);
  c->extra_launches += 9;
}

template <typename T> GraphExec<T>*& graph_of(stagger_ctx* c);
template <> GraphExec<float>*& graph_of<float>(stagger_ctx* c) { return c->g32; }
template <> GraphExec<double>*& graph_of<double>(stagger_ctx* c) { return c->g64; }
template <typename T> T*& work_of(stagger_ctx* c);
template <> float*& work_of<float>(stagger_ctx* c) { return c->w32; }
template <> double*& work_of<double>(stagger_ctx* c) { return c->w64; }

template <typename T>
static int ensure_graph(stagger_ctx* c, bool grads) {
  GraphExec<T>*& G = graph_of<T>(c);
  if (G && (!grads || G->grads)) return STAGGER_OK;
  if (!G) {
    G = new (std::nothrow) GraphExec<T>();
    if (!G) return STAGGER_EOOM;
  }
  return G->init(c->gdef, c->geo, grads);
}

template <typename T>
static int ensure_work(stagger_ctx* c) {
  T*& w = work_of<T>(c);
  if (w) return STAGGER_OK;
  // f1, f2, q, fbar, qbar, and the fixed state, cotangent-in and cotangent-out
  // buffers of the captured adjoint (8 arrays each).
  if (cudaMalloc(&w, sizeof(T) * 64 * (size_t)c->geo.n) != cudaSuccess) {
    w = nullptr;
    return STAGGER_EOOM;
  }
  return STAGGER_OK;
}

template <typename T>
static void lin2(stagger_ctx* c, T* o, const T* x, double a, const T* y, double b, cudaStream_t s) {
  long long n = c->geo.n;
  k_lin2<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(o, x, (T)a, y, (T)b, n);
  ++c->extra_launches;
}
// The same over the eight fields in one launch: o[k] = a x[k] + b y[k], or
// with st >= 0 the coefficient beta_st dt of y read on the device.
template <typename T>
static void lin2x8(stagger_ctx* c, T* const o[8], T* const x[8], double a, T* const y[8],
                   double b, int st, cudaStream_t s) {
  const long long n = c->geo.n;
  Lin8<T> p;
  int vec = n % 4 == 0;
  for (int k = 0; k < 8; ++k) {
    p.o[k] = o[k];
    p.x[k] = x[k];
    p.y[k] = y[k];
    vec &= (((uintptr_t)o[k] | (uintptr_t)x[k] | (uintptr_t)y[k]) & 15) == 0;
  }
  const T* bdt = nullptr;
  if (st >= 0) {
    if constexpr (sizeof(T) == sizeof(float)) bdt = c->bdtf + st;
    else bdt = c->dtp + 1 + st;
  }
  const long long work = vec ? n / 4 : n;
  const unsigned bx = (unsigned)std::min<long long>((work + 255) / 256, 4096);
  k_lin2x8<T><<<dim3(bx, 8), 256, 0, s>>>(p, (T)a, (T)b, bdt, n, vec);
  ++c->extra_launches;
}


template <typename T>
static int graph_rhs(stagger_ctx* c, T* const f[8], T* out[8], cudaStream_t s) {
  int rc = ensure_graph<T>(c, false);
  if (rc) return rc;
  GraphExec<T>* G = graph_of<T>(c);
  const bool rigid = c->params.zwalls == 2, open = c->params.zwalls == 3;
  if (rigid) rigid_fill_g<T>(c, f, s);
  if (open && (rc = open_fill_g<T>(c, f, s))) return rc;
  rc = G->forward(f, s);
  if (rc) return rc;
  long long n = c->geo.n;
  for (int k = 0; k < 8; ++k) {
    k_copy<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out[k], G->output(k), n);
    ++c->extra_launches;
    if (rigid) rigid_zero_g<T>(c, out[k], s);
  }
  if (open) open_rates_g<T>(c, f, out, s);
  STG_CUDA_OK(cudaGetLastError());
  return STAGGER_OK;
}

// One fixed-dt RK3 step through the graph, in place on f.
template <typename T>
static int graph_step(stagger_ctx* c, T* f[8], double dt, cudaStream_t s) {
  int rc = ensure_graph<T>(c, false);
  if (rc) return rc;
  rc = ensure_work<T>(c);
  if (rc) return rc;
  GraphExec<T>* G = graph_of<T>(c);
  T* w = work_of<T>(c);
  const long long n = c->geo.n;
  T* q[8];
  for (int k = 0; k < 8; ++k) q[k] = w + (size_t)k * n;
  const bool rigid = c->params.zwalls == 2, open = c->params.zwalls == 3;
  for (int st = 0; st < 3; ++st) {
    if (rigid) rigid_fill_g<T>(c, f, s);
    if (open && (rc = open_fill_g<T>(c, f, s))) return rc;
    rc = G->forward(f, s);
    if (rc) return rc;
    if (open) {
      T* Fo[8];
      for (int k = 0; k < 8; ++k) Fo[k] = G->output(k);
      open_rates_g<T>(c, f, Fo, s);
    }
    for (int k = 0; k < 8; ++k) {
      if (rigid) rigid_zero_g<T>(c, G->output(k), s);
      if (st == 0) lin2<T>(c, q[k], G->output(k), 1.0, G->output(k), 0.0, s);
      else lin2<T>(c, q[k], q[k], RK_ALPHA[st], G->output(k), 1.0, s);
      lin2<T>(c, f[k], f[k], 1.0, q[k], RK_BETA[st] * dt, s);
    }
  }
  if (rigid) rigid_fill_g<T>(c, f, s);
  if (open && (rc = open_fill_g<T>(c, f, s))) return rc;
  STG_CUDA_OK(cudaGetLastError());
  return STAGGER_OK;
}

// F(f) into out[8] for the stage recompute of the adjoint.
template <typename T>
static int stage_rhs(stagger_ctx* c, GraphExec<T>* G, T* const f[8], T* out[8], cudaStream_t s);
template <>
int stage_rhs<float>(stagger_ctx* c, GraphExec<float>*, float* const f[8], float* out[8],
                     cudaStream_t s) {
  return fused_rhs(c->fused, f, out, s);
}
template <>
int stage_rhs<double>(stagger_ctx* c, GraphExec<double>* G, double* const f[8], double* out[8],
                      cudaStream_t s) {
  int rc = G->forward(f, s);
  if (rc) return rc;
  for (int k = 0; k < 8; ++k) lin2<double>(c, out[k], G->output(k), 1.0, G->output(k), 0.0, s);
  return STAGGER_OK;
}

// Adjoint of one fixed-dt step (see stagger_step_adjoint).
// The adjoint of one step on its workspace, with dt read from c->dtp: the
// body that the adjoint replays as a captured CUDA graph (see below).
template <typename T>
static int adjoint_body(stagger_ctx* c, T* const f0[8], T* const lam_in[8], T* lam_out[8],
                        cudaStream_t s) {
  GraphExec<T>* G = graph_of<T>(c);
  T* w = work_of<T>(c);
  const long long n = c->geo.n;
  T *f1[8], *f2[8], *q[8], *fb[8], *qb[8];
  for (int k = 0; k < 8; ++k) {
    f1[k] = w + (size_t)(0 + k) * n;
    f2[k] = w + (size_t)(8 + k) * n;
    q[k] = w + (size_t)(16 + k) * n;
    fb[k] = w + (size_t)(24 + k) * n;
    qb[k] = w + (size_t)(32 + k) * n;
  }
  const double* A = RK_ALPHA;
  int rc;
  // Recompute the stage states f1, f2 (eqs. (ddt), (tupdate)); the FP32
  // path takes F from the fused kernels, FP64 from the graph.
  if ((rc = stage_rhs<T>(c, G, f0, fb, s))) return rc;
  lin2x8<T>(c, q, fb, 1.0, fb, 0.0, -1, s);
  lin2x8<T>(c, f1, f0, 1.0, q, 0.0, 0, s);
  if ((rc = stage_rhs<T>(c, G, f1, fb, s))) return rc;
  lin2x8<T>(c, q, q, A[1], fb, 1.0, -1, s);
  lin2x8<T>(c, f2, f1, 1.0, q, 0.0, 1, s);
  // Reverse sweep: fbar_3 = lam; qbar_3 = beta_3 dt fbar.
  lin2x8<T>(c, fb, lam_in, 1.0, lam_in, 0.0, -1, s);
  lin2x8<T>(c, qb, fb, 0.0, fb, 0.0, 2, s);
  T* const* stages[3] = {f0, f1, f2};
  for (int st = 2; st >= 0; --st) {
    if ((rc = G->forward(stages[st], s))) return rc;
    if ((rc = G->backward(qb, fb, s))) return rc;     // fbar += J(f_st)^T qbar
    if (st > 0)                                         // qbar_{st} = alpha qbar + beta dt fbar
      lin2x8<T>(c, qb, qb, A[st], fb, 0.0, st - 1, s);
  }
  lin2x8<T>(c, lam_out, fb, 1.0, fb, 0.0, -1, s);
  STG_CUDA_OK(cudaGetLastError());
  return STAGGER_OK;
}

// Adjoint of one fixed-dt step (see stagger_step_adjoint).  The first call
// captures adjoint_body on fixed workspace buffers into a CUDA graph (about
// 4000 launches); every call copies the state and cotangent in, replays the
// graph on the caller's stream, and copies the result out.  If capture is not
// available the body is launched directly (the same kernels).
template <typename T>
static int graph_step_adjoint(stagger_ctx* c, T* const f0[8], double dt, T* const lam_in[8],
                              T* lam_out[8], cudaStream_t s) {
  int rc = ensure_graph<T>(c, true);
  if (rc) return rc;
  // The graph's sweeps on several streams: captured below as a DAG whose
  // independent node kernels overlap.
  rc = graph_of<T>(c)->enable_concurrency();
  if (rc) return rc;
  rc = ensure_work<T>(c);
  if (rc) return rc;
  if (!c->dtp && cudaMalloc(&c->dtp, sizeof(double) * 4) != cudaSuccess) {
    c->dtp = nullptr;
    return STAGGER_EOOM;
  }
  if (!c->bdtf && cudaMalloc(&c->bdtf, sizeof(float) * 4) != cudaSuccess) {
    c->bdtf = nullptr;
    return STAGGER_EOOM;
  }
  k_set_dt3<<<1, 1, 0, s>>>(c->dtp, c->bdtf, dt, RK_BETA[0], RK_BETA[1], RK_BETA[2]);
  ++c->extra_launches;
  const int pi = sizeof(T) == sizeof(float) ? 0 : 1;
  const long long n = c->geo.n;
  T* w = work_of<T>(c);
  T *f0c[8], *lin[8], *lout[8];
  for (int k = 0; k < 8; ++k) {
    f0c[k] = w + (size_t)(40 + k) * n;
    lin[k] = w + (size_t)(48 + k) * n;
    lout[k] = w + (size_t)(56 + k) * n;
  }
  if (c->adj_state[pi] == 0) {
    c->adj_state[pi] = -1;
    if (c->cap || cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) == cudaSuccess) {
      const int timing = c->fused.timing;
      c->fused.timing = 0;   // no event records inside the graph
      const long long before = stagger_launch_count(c);
      cudaGraph_t graph = nullptr;
      if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const int brc = adjoint_body<T>(c, f0c, lin, lout, c->cap);
        const cudaError_t ec = cudaStreamEndCapture(c->cap, &graph);
        if (brc == STAGGER_OK && ec == cudaSuccess && graph &&
            cudaGraphInstantiate(&c->adj_exec[pi], graph, 0) == cudaSuccess)
          c->adj_state[pi] = 1;
        if (graph) cudaGraphDestroy(graph);
      }
      cudaGetLastError();   // a failed capture leaves no sticky error
      // Captured launches have not run: count them per replay instead.
      c->adj_launches[pi] = stagger_launch_count(c) - before;
      c->extra_launches -= c->adj_launches[pi];
      c->fused.timing = timing;
    }
  }
  if (c->adj_state[pi] != 1) return adjoint_body<T>(c, f0, lam_in, lam_out, s);
  const size_t bytes = sizeof(T) * (size_t)n;
  for (int k = 0; k < 8; ++k) {
    STG_CUDA_OK(cudaMemcpyAsync(f0c[k], f0[k], bytes, cudaMemcpyDeviceToDevice, s));
    STG_CUDA_OK(cudaMemcpyAsync(lin[k], lam_in[k], bytes, cudaMemcpyDeviceToDevice, s));
  }
  STG_CUDA_OK(cudaGraphLaunch(c->adj_exec[pi], s));
  c->extra_launches += c->adj_launches[pi];
  for (int k = 0; k < 8; ++k)
    STG_CUDA_OK(cudaMemcpyAsync(lam_out[k], lout[k], bytes, cudaMemcpyDeviceToDevice, s));
  return STAGGER_OK;
}

extern "C" {

int stagger_step_adjoint(stagger_ctx* c, float* const state_n[8], double dt,
                         float* const lam_np1[8], float* lam_n[8], void* stream) {
  if (!c || !ptrs_ok((void* const*)state_n) || !ptrs_ok((void* const*)lam_np1) ||
      !ptrs_ok((void* const*)lam_n) || !(dt > 0))
    return STAGGER_EINVAL;
  // the op graph has no transpose of the wall fills
  if (c->params.zwalls) return STAGGER_EUNSUPPORTED;
  return graph_step_adjoint<float>(c, state_n, dt, lam_np1, lam_n, (cudaStream_t)stream);
}

int stagger_rhs_unfused(stagger_ctx* c, float* const state[8], float* dfdt[8], void* stream) {
  if (!c || !ptrs_ok((void* const*)state) || !ptrs_ok((void* const*)dfdt)) return STAGGER_EINVAL;
  if (c->params.zwalls == 1) return STAGGER_EUNSUPPORTED;   // the graph does not reflect
  if (c->params.zwalls == 3 && c->params.top_tpot > 0) return STAGGER_EUNSUPPORTED;
  return graph_rhs<float>(c, state, dfdt, (cudaStream_t)stream);
}

int stagger_rhs_unfused_f64(stagger_ctx* c, double* const state[8], double* dfdt[8],
                            void* stream) {
  if (!c || !ptrs_ok((void* const*)state) || !ptrs_ok((void* const*)dfdt)) return STAGGER_EINVAL;
  if (c->params.zwalls == 1) return STAGGER_EUNSUPPORTED;   // the graph does not reflect
  if (c->params.zwalls == 3 && c->params.top_tpot > 0) return STAGGER_EUNSUPPORTED;
  return graph_rhs<double>(c, state, dfdt, (cudaStream_t)stream);
}

int stagger_step_unfused_f64(stagger_ctx* c, double* state[8], double dt, void* stream) {
  if (!c || !ptrs_ok((void* const*)state) || !(dt > 0)) return STAGGER_EINVAL;
  if (c->params.zwalls == 1) return STAGGER_EUNSUPPORTED;   // the graph does not reflect
  if (c->params.zwalls == 3 && c->params.top_tpot > 0) return STAGGER_EUNSUPPORTED;
  return graph_step<double>(c, state, dt, (cudaStream_t)stream);
}

int stagger_step_adjoint_f64(stagger_ctx* c, double* const state_n[8], double dt,
                             double* const lam_np1[8], double* lam_n[8], void* stream) {
  if (!c || !ptrs_ok((void* const*)state_n) || !ptrs_ok((void* const*)lam_np1) ||
      !ptrs_ok((void* const*)lam_n) || !(dt > 0))
    return STAGGER_EINVAL;
  // the op graph has no transpose of the wall fills
  if (c->params.zwalls) return STAGGER_EUNSUPPORTED;
  return graph_step_adjoint<double>(c, state_n, dt, lam_np1, lam_n, (cudaStream_t)stream);
}

int stagger_step_host(stagger_ctx* c, float* state_host[8], int nsteps, double dt, void* stream) {
  if (!c || !ptrs_ok((void* const*)state_host) || nsteps < 0 || !(dt == dt)) return STAGGER_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)c->geo.n;
  if (!c->host_state) {
    if (cudaMalloc(&c->host_state, sizeof(float) * 8 * n) != cudaSuccess) {
      c->host_state = nullptr;
      return STAGGER_EOOM;
    }
  }
  float* d[8];
  for (int k = 0; k < 8; ++k) {
    d[k] = c->host_state + k * n;
    STG_CUDA_OK(cudaMemcpyAsync(d[k], state_host[k], sizeof(float) * n, cudaMemcpyHostToDevice, s));
  }
  for (int i = 0; i < nsteps; ++i) {
    int rc = fused_step_graphed(c->fused, d, dt, s);
    if (rc) return rc;
  }
  for (int k = 0; k < 8; ++k)
    STG_CUDA_OK(cudaMemcpyAsync(state_host[k], d[k], sizeof(float) * n, cudaMemcpyDeviceToHost, s));
  STG_CUDA_OK(cudaStreamSynchronize(s));
  return STAGGER_OK;
}

}  // extern "C"
