// dword_probe.cu -- test driver for the double-word primitives of
// paper_1908_03972_gb300/csrc/dword.cuh (built and run by
// tests/test_gpu_dword.py; not part of the library).
//
// Input: n, then n pairs (a, b) of binary64 values (raw little-endian).
// Output per pair: the (h, l) FP32 words of x = dw(a), y = dw(b), x + y,
// x - y, x * y, 1 / y, sqrt(|x|) and the Dot2 sum x y + y y - x x + y, then
// dw_to_double(x) as one binary64 value.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../paper_1908_03972_gb300/csrc/dword.cuh"

using pmg::dw;

__global__ void probe(int n, const double* a, const double* b, float* out, double* back) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const dw x = pmg::dw_from_double(a[i]), y = pmg::dw_from_double(b[i]);
  pmg::dw_acc acc;
  acc.add_prod(x, y);
  acc.add_prod(y, y);
  acc.add_prod(-x, x);
  acc.add(y);
  const dw r[8] = {x, y, x + y, x - y, x * y, pmg::rcp(y), pmg::sqrt_dw(pmg::abs_dw(x)), acc.value()};
  for (int k = 0; k < 8; ++k) {
    out[(size_t)i * 16 + 2 * k] = r[k].h;
    out[(size_t)i * 16 + 2 * k + 1] = r[k].l;
  }
  back[i] = pmg::dw_to_double(x);
}

int main(int argc, char** argv) {
  if (argc != 3) {
    fprintf(stderr, "usage: dword_probe in.bin out.bin\n");
    return 2;
  }
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 3;
  int n = 0;
  if (fread(&n, sizeof(int), 1, f) != 1 || n <= 0 || n > (1 << 20)) return 4;
  std::vector<double> a(n), b(n);
  if (fread(a.data(), sizeof(double), n, f) != (size_t)n || fread(b.data(), sizeof(double), n, f) != (size_t)n)
    return 5;
  fclose(f);
  double *da, *db, *dback;
  float* dout;
  if (cudaMalloc(&da, n * sizeof(double)) != cudaSuccess || cudaMalloc(&db, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dback, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dout, (size_t)n * 16 * sizeof(float)) != cudaSuccess)
    return 6;
  cudaMemcpy(da, a.data(), n * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(db, b.data(), n * sizeof(double), cudaMemcpyHostToDevice);
  probe<<<(n + 127) / 128, 128>>>(n, da, db, dout, dback);
  std::vector<float> out((size_t)n * 16);
  std::vector<double> back(n);
  cudaMemcpy(out.data(), dout, out.size() * sizeof(float), cudaMemcpyDeviceToHost);
  cudaMemcpy(back.data(), dback, n * sizeof(double), cudaMemcpyDeviceToHost);
  const cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    fprintf(stderr, "CUDA error: %s\n", cudaGetErrorString(e));
    return 7;
  }
  FILE* g = fopen(argv[2], "wb");
  if (!g) return 8;
  fwrite(out.data(), sizeof(float), out.size(), g);
  fwrite(back.data(), sizeof(double), back.size(), g);
  fclose(g);
  return 0;
}
