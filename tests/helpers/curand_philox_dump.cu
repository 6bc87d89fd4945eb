// Independent Philox4x32-10 on the GPU: cuRAND's curand_Philox4x32_10 device
// routine (from the CUDA toolkit headers), used to pin both the oracle's
// generator and the library's.  Reads lines "c0 c1 c2 c3 k0 k1" from stdin and
// prints the four output words of each.
#include <cstdio>
#include <vector>

#include <curand_kernel.h>

__global__ void run(const uint4 *ctr, const uint2 *key, uint4 *out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

int main() {
  std::vector<uint4> c;
  std::vector<uint2> k;
  unsigned a, b, d, e, f, g;
  while (std::scanf("%u %u %u %u %u %u", &a, &b, &d, &e, &f, &g) == 6) {
    c.push_back(make_uint4(a, b, d, e));
    k.push_back(make_uint2(f, g));
  }
  const int n = static_cast<int>(c.size());
  if (n == 0) return 0;
  uint4 *dc, *dout;
  uint2 *dk;
  if (cudaMalloc(&dc, n * sizeof(uint4)) != cudaSuccess) return 2;
  if (cudaMalloc(&dk, n * sizeof(uint2)) != cudaSuccess) return 2;
  if (cudaMalloc(&dout, n * sizeof(uint4)) != cudaSuccess) return 2;
  cudaMemcpy(dc, c.data(), n * sizeof(uint4), cudaMemcpyHostToDevice);
  cudaMemcpy(dk, k.data(), n * sizeof(uint2), cudaMemcpyHostToDevice);
  run<<<(n + 255) / 256, 256>>>(dc, dk, dout, n);
  std::vector<uint4> out(n);
  if (cudaMemcpy(out.data(), dout, n * sizeof(uint4), cudaMemcpyDeviceToHost) != cudaSuccess)
    return 3;
  for (int i = 0; i < n; ++i) std::printf("%u %u %u %u\n", out[i].x, out[i].y, out[i].z, out[i].w);
  cudaFree(dc);
  cudaFree(dk);
  cudaFree(dout);
  return 0;
}
