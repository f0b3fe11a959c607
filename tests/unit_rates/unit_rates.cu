// Throughput of the integer instructions the walk kernels are built from, in
// lane-operations per SM per clock on the current GPU: the unit counts behind
// the roofline denominators (population counts on the XU pipe, LOP3 and IMAD
// on the ALU and FMA pipes).  Every lane runs 8 independent dependency chains
// of one instruction kind written as inline PTX whose results feed the next
// instruction, so the compiler cannot fold them; per-SM cycle counts come from
// clock64() of the blocks resident on each SM.  All accesses are in bounds and
// nothing waits on anything.  Prints one "name value" line per instruction.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <vector>

#define CHAINS 8
#define ITER 2048

template <int OP>
__global__ void probe(uint32_t seed, uint32_t *sink, unsigned long long *rec) {
  uint32_t x[CHAINS], z[CHAINS];
  const uint32_t y = seed ^ threadIdx.x;
  float f[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) {
    x[c] = seed * (c + 1) + threadIdx.x;
    z[c] = x[c] * 7u + 1u;
    f[c] = (float)x[c];
  }
  const unsigned long long t0 = clock64();
  for (int it = 0; it < ITER; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) {
        if (OP == 0) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[c]) : "r"(y), "r"(z[c]));
        if (OP == 1) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(y), "r"(z[c]));
        if (OP == 2) asm volatile("shf.r.wrap.b32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(z[c]), "r"(y));
        if (OP == 3) asm volatile("popc.b32 %0, %0;" : "+r"(x[c]));
        if (OP == 4) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[c]) : "f"(1.0001f), "f"(0.5f));
        if (OP == 5) asm volatile("dp4a.s32.s32 %0, %1, %2, %0;" : "+r"(x[c]) : "r"(y), "r"(z[c]));
        if (OP == 6) x[c] = __shfl_sync(0xffffffffu, x[c], (threadIdx.x + c) & 31);
        if (OP == 7) {  // one POPC and one LOP3 per chain step
          asm volatile("popc.b32 %0, %0;" : "+r"(x[c]));
          asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(z[c]) : "r"(y), "r"(x[c]));
        }
        if (OP == 8) {  // one POPC and three LOP3 per chain step
          asm volatile("popc.b32 %0, %0;" : "+r"(x[c]));
          asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(z[c]) : "r"(y), "r"(x[c]));
          asm volatile("lop3.b32 %0, %0, %1, %2, 0xe8;" : "+r"(z[c]) : "r"(y), "r"(x[c]));
          asm volatile("lop3.b32 %0, %0, %1, %2, 0x6a;" : "+r"(z[c]) : "r"(y), "r"(x[c]));
        }
        if (OP == 9) {  // one LOP3 and one IMAD per chain step
          asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[c]) : "r"(y), "r"(z[c]));
          asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(z[c]) : "r"(y), "r"(x[c]));
        }
      }
    }
  }
  const unsigned long long t1 = clock64();
  uint32_t acc = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) acc += x[c] + z[c] + __float_as_uint(f[c]);
  if (acc == 0x12345678u) sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
  __shared__ unsigned long long tmin, tmax;
  if (threadIdx.x == 0) {
    tmin = ~0ull;
    tmax = 0;
  }
  __syncthreads();
  atomicMin(&tmin, t0);
  atomicMax(&tmax, t1);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    rec[blockIdx.x * 3 + 0] = smid;
    rec[blockIdx.x * 3 + 1] = tmin;
    rec[blockIdx.x * 3 + 2] = tmax;
  }
}

template <int OP>
static void run(const char *name, int ops_per_step, int nsm) {
  const int bps = 4, tpb = 256, nb = nsm * bps;
  uint32_t *sink;
  unsigned long long *rec;
  cudaMalloc(&sink, sizeof(uint32_t) * nb * tpb);
  cudaMalloc(&rec, sizeof(unsigned long long) * nb * 3);
  probe<OP><<<nb, tpb>>>(12345u, sink, rec);  // warm-up
  probe<OP><<<nb, tpb>>>(12345u, sink, rec);
  std::vector<unsigned long long> h(nb * 3);
  cudaMemcpy(h.data(), rec, sizeof(unsigned long long) * nb * 3, cudaMemcpyDeviceToHost);
  std::vector<unsigned long long> lo(4096, ~0ull), hi(4096, 0);
  std::vector<int> cnt(4096, 0);
  for (int b = 0; b < nb; ++b) {
    const int s = (int)h[b * 3];
    if (s < 4096) {
      cnt[s]++;
      lo[s] = std::min(lo[s], h[b * 3 + 1]);
      hi[s] = std::max(hi[s], h[b * 3 + 2]);
    }
  }
  const double per_block = (double)ITER * 4 * CHAINS * ops_per_step * tpb;
  double sum = 0;
  int sms = 0;
  for (int s = 0; s < 4096; ++s)
    if (cnt[s]) {
      sum += per_block * cnt[s] / (double)(hi[s] - lo[s]);
      ++sms;
    }
  printf("%s %.4f %d\n", name, sum / sms, sms);
  cudaFree(sink);
  cudaFree(rec);
}

int main() {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, 0) != cudaSuccess) {
    printf("no CUDA device\n");
    return 1;
  }
  printf("device %d.%d %d\n", p.major, p.minor, p.multiProcessorCount);
  const int n = p.multiProcessorCount;
  run<0>("LOP3", 1, n);
  run<1>("IMAD", 1, n);
  run<3>("POPC", 1, n);
  run<7>("POPC+LOP3", 2, n);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
