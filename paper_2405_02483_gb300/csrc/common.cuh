// Shared device helpers of libstagger: mesh geometry, periodic indexing,
// the staggered operator weights of eqs. (deriv)/(interp), and error macros.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/stagger.h"

namespace stg {

// Interpolation weights, eq. (interpcoef): a = 1/2 - b - c.
#define STG_IA (150.0 / 256.0)
#define STG_IB (-25.0 / 256.0)
#define STG_IC (3.0 / 256.0)
// Derivative weights, eq. (derivcoef): c = 3/640, b = -25/384, a = 1 - 3b - 5c.
#define STG_DA (225.0 / 192.0)
#define STG_DB (-25.0 / 384.0)
#define STG_DC (3.0 / 640.0)

// Low-storage RK3 constants, eq. (tconst), as printed.
static const double RK_ALPHA[3] = {0.0, -0.641874, -1.31021};
static const double RK_BETA[3] = {0.46173, 0.924087, 0.390614};

struct Geo {
  int nx, ny, nz;
  long long sy;   // stride of y (= nx)
  long long sz;   // stride of z (= nx*ny)
  long long n;    // cells
};

inline Geo make_geo(int nx, int ny, int nz) {
  Geo g;
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.sy = nx; g.sz = (long long)nx * ny; g.n = g.sz * nz;
  return g;
}

// Periodic wrap of j into [0, n).  Fast path for the usual |offset| < n.
__host__ __device__ __forceinline__ int wrap(int j, int n) {
  if (j >= 0 && j < n) return j;
  if (j < 0 && j >= -n) return j + n;
  if (j >= n && j < 2 * n) return j - n;
  j %= n;
  return j < 0 ? j + n : j;
}

// Linear index of (i+di, j+dj, k+dk) with periodic wrap.
__host__ __device__ __forceinline__ long long lin(const Geo& g, int i, int j, int k) {
  return (long long)k * g.sz + (long long)j * g.sy + i;
}

// Grid and parameter checks of stagger_create (STAGGER_OK or STAGGER_EINVAL).
int validate_inputs(const stagger_grid* g, const stagger_params* p);

}  // namespace stg

#define STG_CUDA_OK(call)                                   \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) { return STAGGER_ECUDA; }        \
  } while (0)
