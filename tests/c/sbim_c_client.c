/*
 * A plain C client of include/sbim.h: no PyTorch, device memory from the CUDA
 * runtime.  It reads a boundary history from a binary file, steps one
 * half-space through it with sbim_step (device buffers) and sbim_step_host
 * (host buffers, on a second handle), and writes every step's traction from
 * both to a binary file, for the test that builds and runs it.
 *
 * usage: sbim_c_client in.bin out.bin
 *   in.bin:  int32 n1, n3, n_cut, side, steps; float64 L1, L3, cs, cp, rho, dt;
 *            then steps x (u, v) as float32 [3][n3][n1] each
 *   out.bin: steps x (tau_device, tau_host) as float32 [3][n3][n1] each
 * Exit status 0 on success; a failing call prints sbim_last_error().
 */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "sbim.h"

#define CHECK(call)                                                          \
  do {                                                                       \
    int rc_ = (call);                                                        \
    if (rc_ != SBIM_OK) {                                                    \
      fprintf(stderr, "%s -> %d: %s\n", #call, rc_, sbim_last_error());      \
      return 2;                                                              \
    }                                                                        \
  } while (0)

#define CUDA(call)                                                           \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      fprintf(stderr, "%s: %s\n", #call, cudaGetErrorString(e_));            \
      return 3;                                                              \
    }                                                                        \
  } while (0)

int main(int argc, char** argv) {
  if (argc != 3) {
    fprintf(stderr, "usage: %s in.bin out.bin\n", argv[0]);
    return 1;
  }
  FILE* in = fopen(argv[1], "rb");
  FILE* out = fopen(argv[2], "wb");
  if (!in || !out) return 1;
  int hdr[5];
  double par[6];
  if (fread(hdr, sizeof(int), 5, in) != 5 || fread(par, sizeof(double), 6, in) != 6) return 1;
  const int n1 = hdr[0], n3 = hdr[1], n_cut = hdr[2], side = hdr[3], steps = hdr[4];
  const size_t count = (size_t)3 * n1 * n3, bytes = count * sizeof(float);

  sbim_handle dev = NULL, host = NULL;
  CHECK(sbim_create(&dev, n1, n3, par[0], par[1], par[2], par[3], par[4], par[5], n_cut, side,
                    SBIM_FP32, 1, NULL));
  CHECK(sbim_create(&host, n1, n3, par[0], par[1], par[2], par[3], par[4], par[5], n_cut, side,
                    SBIM_FP32, 1, NULL));
  float *u = (float*)malloc(bytes), *v = (float*)malloc(bytes), *t = (float*)malloc(bytes);
  float *du, *dv, *dt;
  CUDA(cudaMalloc((void**)&du, bytes));
  CUDA(cudaMalloc((void**)&dv, bytes));
  CUDA(cudaMalloc((void**)&dt, bytes));
  for (int n = 0; n < steps; ++n) {
    if (fread(u, 1, bytes, in) != bytes || fread(v, 1, bytes, in) != bytes) return 1;
    CUDA(cudaMemcpy(du, u, bytes, cudaMemcpyHostToDevice));
    CUDA(cudaMemcpy(dv, v, bytes, cudaMemcpyHostToDevice));
    CHECK(sbim_step(dev, du, dv, dt));
    CUDA(cudaMemcpy(t, dt, bytes, cudaMemcpyDeviceToHost));   /* legacy stream: ordered */
    fwrite(t, 1, bytes, out);
    CHECK(sbim_step_host(host, u, v, t));
    fwrite(t, 1, bytes, out);
  }
  CHECK(sbim_check_device(dev));
  long long n = 0;
  CHECK(sbim_get_step(dev, &n));
  if (n != steps) return 4;
  CHECK(sbim_destroy(dev));
  CHECK(sbim_destroy(host));
  cudaFree(du);
  cudaFree(dv);
  cudaFree(dt);
  free(u);
  free(v);
  free(t);
  fclose(in);
  fclose(out);
  return 0;
}
