/* A plain C user of libstagger: builds a smooth 16^3 MHD state in host
 * memory, takes two fixed-dt steps through stagger_step_host (the library
 * copies to and from the device), and writes the eight fields to a binary
 * file.  No CUDA runtime and no Python: only include/stagger.h and the
 * library.  Usage: c_abi_step OUT.bin */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "stagger.h"

int main(int argc, char** argv) {
  if (argc != 2) {
    fprintf(stderr, "usage: %s OUT.bin\n", argv[0]);
    return 2;
  }
  const int n = 16;
  const size_t cells = (size_t)n * n * n;
  const double h = 1.0 / n, tau = 6.283185307179586;
  stagger_grid grid = {n, n, n, h, h, h};
  stagger_params p;
  if (stagger_params_default(&p) != STAGGER_OK) return 3;
  p.nu1 = 0.04; p.nu2 = 1.0; p.nu3 = 0.04; p.do_quench = 1;
  p.ref[0] = 1.0;       /* rho = 1 + stored */
  p.ref[4] = 0.9;       /* E = 0.9 + stored */
  p.ref[7] = 0.3;       /* Bz = 0.3 + stored */
  float* f[8];
  for (int c = 0; c < 8; ++c) {
    f[c] = (float*)calloc(cells, sizeof(float));
    if (!f[c]) return 4;
  }
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const size_t c = ((size_t)k * n + j) * n + i;
        const double x = (i + 0.5) * h, y = (j + 0.5) * h, z = (k + 0.5) * h;
        f[0][c] = (float)(0.02 * sin(tau * x) * cos(tau * z));
        f[1][c] = (float)(0.1 * sin(tau * y));
        f[2][c] = (float)(0.1 * sin(tau * z));
        f[3][c] = (float)(0.1 * sin(tau * x));
        f[4][c] = (float)(0.01 * cos(tau * y));
        f[5][c] = (float)(0.05 * cos(tau * z));
        f[6][c] = (float)(0.05 * cos(tau * x));
      }
  stagger_ctx* ctx = NULL;
  int st = stagger_create(&grid, &p, &ctx);
  if (st != STAGGER_OK) {
    fprintf(stderr, "stagger_create: %s\n", stagger_strerror(st));
    return 5;
  }
  st = stagger_step_host(ctx, f, 2, 1e-3, NULL);
  if (st != STAGGER_OK) {
    fprintf(stderr, "stagger_step_host: %s\n", stagger_strerror(st));
    return 6;
  }
  stagger_destroy(ctx);
  FILE* out = fopen(argv[1], "wb");
  if (!out) return 7;
  for (int c = 0; c < 8; ++c) fwrite(f[c], sizeof(float), cells, out);
  fclose(out);
  for (int c = 0; c < 8; ++c) free(f[c]);
  printf("ok\n");
  return 0;
}
