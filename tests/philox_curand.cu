// Test helper: Philox4x32-10 from cuRAND's public device header, so the
// oracle's own Philox can be checked against an independent implementation.
// Reads n records of (c0, c1, c2, c3, k0, k1) uint32 from argv[1], writes n
// records of (r0, r1, r2, r3) uint32 to argv[2].
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include <curand_kernel.h>

__global__ void k_philox(const uint32_t* in, uint32_t* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t* q = in + 6 * i;
  const uint4 r = curand_Philox4x32_10(make_uint4(q[0], q[1], q[2], q[3]), make_uint2(q[4], q[5]));
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 3;
  std::vector<uint32_t> in;
  uint32_t w;
  while (fread(&w, 4, 1, f) == 1) in.push_back(w);
  fclose(f);
  const int n = (int)(in.size() / 6);
  uint32_t *d_in = nullptr, *d_out = nullptr;
  if (cudaMalloc(&d_in, in.size() * 4) != cudaSuccess) return 4;
  if (cudaMalloc(&d_out, (size_t)n * 16) != cudaSuccess) return 4;
  cudaMemcpy(d_in, in.data(), in.size() * 4, cudaMemcpyHostToDevice);
  k_philox<<<(n + 255) / 256, 256>>>(d_in, d_out, n);
  std::vector<uint32_t> out((size_t)n * 4);
  if (cudaMemcpy(out.data(), d_out, out.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return 5;
  FILE* g = fopen(argv[2], "wb");
  if (!g) return 3;
  fwrite(out.data(), 4, out.size(), g);
  fclose(g);
  cudaFree(d_in);
  cudaFree(d_out);
  return 0;
}
