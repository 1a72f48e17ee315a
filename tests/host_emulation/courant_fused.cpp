// Host build of the fused kernels: the Courant maxima taken inside the
// stage-1 kernels (wave speed in k_nu_raw, <nu> in k_nu_maxsmooth, rate in the
// mass and energy k_div) equal those of the separate pass k_courant_part, bit
// for bit.  Threads of a block run one at a time, and every block twice: a
// warp shuffle returns the running maximum, over the lanes of its warp that
// have run, of the same reduction; the first pass completes the block's
// shared-memory partials and the second, whose atomics alone take effect,
// reads them (every other write these kernels make is idempotent), so each
// block's reduction sees all of its threads as on the device.  Exit status: the
// number of shapes that differ.
#include <cuda_runtime.h>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
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
static inline float rsqrtf(float x) { return 1.f / sqrtf(x); }
static inline float __uint_as_float(unsigned u) { float f; memcpy(&f, &u, 4); return f; }
static inline unsigned __float_as_uint(float f) { unsigned u; memcpy(&u, &f, 4); return u; }
static inline unsigned max(unsigned a, unsigned b) { return a > b ? a : b; }
static inline int min(int a, int b) { return a < b ? a : b; }
// Running maximum per (block, warp, reduction): a reduction is five shuffles
// (offsets 16 .. 1), and CALLS counts a thread's shuffles since it started.
static std::map<long long, unsigned> WARP_ACC;
static int CALLS = 0;
static inline unsigned __shfl_xor_sync(unsigned, unsigned v, int) {
  const long long b = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
  const int seq = CALLS++ / 5;
  unsigned& a = WARP_ACC[(b * 64 + tid / 32) * 16 + seq];
  a = max(a, v);
  return a;
}
static int PASS = 1;   // atomics take effect in the second pass only
static inline unsigned atomicMax(unsigned* p, unsigned v) {
  unsigned o = *p;
  if (PASS == 1 && v > o) *p = v;
  return o;
}
#include "../../paper_2405_02483_gb300/csrc/fused_kernels.cuh"
using namespace stg;

template <class K>
static void run(dim3 gd, dim3 bd, K kern) {
  gridDim = gd;
  blockDim = bd;
  WARP_ACC.clear();
  for (unsigned bz = 0; bz < gd.z; ++bz)
    for (unsigned by = 0; by < gd.y; ++by)
      for (unsigned bx = 0; bx < gd.x; ++bx)
        for (PASS = 0; PASS < 2; ++PASS)
          for (int tz = bd.z - 1; tz >= 0; --tz)
            for (int ty = bd.y - 1; ty >= 0; --ty)
              for (int tx = bd.x - 1; tx >= 0; --tx) {
                blockIdx = make_uint3(bx, by, bz);
                threadIdx = make_uint3(tx, ty, tz);
                CALLS = 0;
                kern();
              }
}

int main() {
  const int shapes[][3] = {{16, 8, 40}, {4, 1, 3}, {132, 6, 5}, {8, 3, 9}, {12, 2, 1}};
  int bad = 0;
  for (const auto& sh : shapes) {
    const int nx = sh[0], ny = sh[1], nz = sh[2];
    const Geo g = make_geo(nx, ny, nz);
    std::mt19937 rng(nx * 11 + nz);
    std::uniform_real_distribution<float> U(-1.f, 1.f);
    auto field = [&](float a) { std::vector<float> v(g.n); for (auto& x : v) x = a * U(rng); return v; };
    std::vector<float> ux = field(1), uy = field(1), uz = field(1), rd = field(0.1f), Ed = field(0.1f),
                       bx = field(0.3f), by = field(0.3f), bz = field(0.3f), px = field(1), py = field(1),
                       pz = field(1), gx = field(1), gy = field(1), gz = field(1), qt = field(1);
    std::vector<float> nv(g.n), nu(g.n), lnu(g.n), q0(g.n), q4(g.n), dummy(g.n);
    KPar k;
    memset(&k, 0, sizeof(k));
    k.ih[0] = nx; k.ih[1] = 1.1f * ny; k.ih[2] = 0.9f * nz;
    k.gamma = 5.f / 3.f; k.gm1 = 2.f / 3.f; k.r0 = 1.f; k.E0 = 1.5f; k.r0pos = 1; k.e0 = 1.5f;
    k.Bref[2] = 0.3f; k.rm = 1; k.visc = 1; k.nu1 = 0.04f; k.nu3 = 0.04f; k.nu2 = 1.f;
    k.nu2dl = 1.f / nx; k.dlmin = 1.f / nx; k.sp[0] = k.sp[1] = k.sp[2] = 1.f / nx;
    const dim3 gg((nx + BX * 4 - 1) / (BX * 4), (ny + BY - 1) / BY, (nz + BZ - 1) / BZ), bb(BX, BY, BZ);
    unsigned fused[3] = {0u, 0u, 0u}, ref[3] = {0u, 0u, 0u};
    run(gg, bb, [&] {
      k_nu_raw<false, true, Nb4>(ux.data(), uy.data(), uz.data(), rd.data(), Ed.data(), bx.data(),
                                 by.data(), bz.data(), nullptr, nullptr, nullptr, nv.data(), fused, k, g);
    });
    const dim3 gm((nx + 127) / 128, (ny + NUZ_TY - 1) / NUZ_TY, (nz + NUZ_ZC - 1) / NUZ_ZC);
    run(gm, dim3(32, NUZ_TY, 1), [&] { k_nu_maxsmooth<true>(nv.data(), nu.data(), lnu.data(), fused + 2, g); });
    DivIn di;
    memset(&di, 0, sizeof(di));
    di.px = px.data(); di.py = py.data(); di.pz = pz.data();
    di.gx = gx.data(); di.gy = gy.data(); di.gz = gz.data(); di.qt = qt.data();
    for (int c = 0; c < 8; ++c) di.f[c] = dummy.data();
    di.f[0] = rd.data();
    di.f[4] = Ed.data();
    float* o = dummy.data();
    float bdtv = 0;
    run(gg, bb, [&] {
      k_div<Nb4, 0x11, true>(di, q0.data(), o, o, o, q4.data(), o, o, o, q0.data(), o, o, o, q4.data(), o,
                             o, o, 0.f, &bdtv, 0, fused + 1, k, g);
    });
    run(gg, bb, [&] {
      k_courant_part<Nb4>(ux.data(), uy.data(), uz.data(), rd.data(), Ed.data(), bx.data(), by.data(),
                          bz.data(), q0.data(), q4.data(), nu.data(), ref, k, g);
    });
    int diff = 0;
    for (int c = 0; c < 3; ++c) diff += fused[c] != ref[c];
    printf("%dx%dx%d: wave %.9g / %.9g, rate %.9g / %.9g, nu %.9g / %.9g, %d differing\n", nx, ny, nz,
           __uint_as_float(fused[0]), __uint_as_float(ref[0]), __uint_as_float(fused[1]),
           __uint_as_float(ref[1]), __uint_as_float(fused[2]), __uint_as_float(ref[2]), diff);
    bad += diff != 0 || ref[0] == 0u || ref[1] == 0u || ref[2] == 0u;
  }
  return bad;
}
