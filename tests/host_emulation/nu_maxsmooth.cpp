// Host build of the fused kernels (CUDA qualifiers mapped to host C++, each
// kernel run over its grid one thread at a time): k_nu_maxsmooth, the
// z-marching 3x3x3 max and mean of the viscosity, must equal k_nu_max followed
// by k_nu_smooth bit for bit, on shapes with partial blocks, single cells
// along an axis and fewer planes than the march's halo.  Exit status: the
// number of shapes that differ.
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
uint3 blockIdx, threadIdx;
dim3 blockDim, gridDim;
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

int main() {
  const int shapes[][3] = {{16, 8, 40}, {4, 1, 3}, {132, 6, 5}, {8, 3, 70}, {12, 2, 1}, {20, 12, 33}};
  int bad = 0;
  for (const auto& sh : shapes) {
    const int nx = sh[0], ny = sh[1], nz = sh[2];
    const Geo g = make_geo(nx, ny, nz);
    std::vector<float> nv(g.n), nm(g.n), nu1(g.n), ln1(g.n), nu2(g.n), ln2(g.n);
    std::mt19937 rng(nx * 7 + nz);
    std::uniform_real_distribution<float> U(0.f, 2.f);
    for (auto& v : nv) v = U(rng) * U(rng);
    const dim3 gg((nx + BX * 4 - 1) / (BX * 4), (ny + BY - 1) / BY, (nz + BZ - 1) / BZ), bb(BX, BY, BZ);
    run(gg, bb, [&] { k_nu_max<Nb4>(nv.data(), nm.data(), g); });
    run(gg, bb, [&] { k_nu_smooth<Nb4, false>(nm.data(), nu1.data(), ln1.data(), nullptr, g); });
    const dim3 gm((nx + 127) / 128, (ny + NUZ_TY - 1) / NUZ_TY, (nz + NUZ_ZC - 1) / NUZ_ZC);
    run(gm, dim3(32, NUZ_TY, 1), [&] { k_nu_maxsmooth<false>(nv.data(), nu2.data(), ln2.data(), nullptr, g); });
    long long diff = 0;
    for (long long i = 0; i < g.n; ++i)
      diff += (memcmp(&nu1[i], &nu2[i], 4) != 0) + (memcmp(&ln1[i], &ln2[i], 4) != 0);
    printf("%dx%dx%d: %lld differing values\n", nx, ny, nz, diff);
    bad += diff != 0;
  }
  return bad;
}
