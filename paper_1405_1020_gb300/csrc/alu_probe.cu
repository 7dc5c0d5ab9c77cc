// alu_probe.cu -- integer-ALU throughput of one GPU, the denominator of the
// filter's roofline (the method's per-pixel work is integer adds, compares,
// masks and shifts).
//
// Every thread runs NCHAIN independent chains of 32-bit integer operations in
// inline PTX, so the issue of one chain never waits for another's result;
// blocks fill every SM.  Two mixes are timed with CUDA events: add/xor
// (IADD3 and LOP3 on the integer pipe) and multiply-add (IMAD).  The result
// is operations per clock per SM, using the SM clock the driver reports as
// the maximum, and the whole-GPU rate at that clock.  The chains' final
// values are written out so that nothing is optimised away.
//
// Build: python -c "from paper_1405_1020_gb300.csrc import build; build.build_alu_probe()"
// Run:   paper_1405_1020_gb300/alu_probe

#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>

namespace {

constexpr int NCHAIN = 8;
constexpr int NITER = 4096;
constexpr int UNROLL = 16;

__global__ void __launch_bounds__(256) add_xor_kernel(unsigned *out, unsigned seed) {
  unsigned a[NCHAIN];
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) a[c] = seed * (threadIdx.x + 1u) + c;
  const unsigned k1 = seed | 1u, k2 = seed ^ 0x9E3779B9u;
  for (int it = 0; it < NITER; ++it) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
      for (int c = 0; c < NCHAIN; ++c) {
        // one add and one xor per chain and step: each depends on the
        // previous, so they cannot be merged into one three-input add
        asm volatile("add.u32 %0, %0, %1;" : "+r"(a[c]) : "r"(k1));
        asm volatile("xor.b32 %0, %0, %1;" : "+r"(a[c]) : "r"(k2));
      }
    }
  }
  unsigned s = 0;
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) s ^= a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) mad_kernel(unsigned *out, unsigned seed) {
  unsigned a[NCHAIN];
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) a[c] = seed * (threadIdx.x + 1u) + c;
  const unsigned k1 = seed | 1u, k2 = seed ^ 0x9E3779B9u;
  for (int it = 0; it < NITER; ++it) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
      for (int c = 0; c < NCHAIN; ++c)
        asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[c]) : "r"(k1), "r"(k2));
    }
  }
  unsigned s = 0;
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) s ^= a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

bool ok(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return true;
  std::fprintf(stderr, "%s: %s\n", what, cudaGetErrorString(e));
  return false;
}

}  // namespace

int main() {
  int dev = 0, sms = 0, clk_khz = 0;
  if (!ok(cudaGetDevice(&dev), "cudaGetDevice")) return 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  const int blocks = sms * 8, threads = 256;
  unsigned *out = nullptr;
  if (!ok(cudaMalloc(&out, sizeof(unsigned) * blocks * threads), "cudaMalloc")) return 1;
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  struct Mix {
    const char *name;
    void (*fn)(unsigned *, unsigned);
    double ops_per_step;  // per chain and unrolled step
  } mixes[2] = {{"add+xor (IADD3/LOP3)", add_xor_kernel, 2.0}, {"mad (IMAD)", mad_kernel, 1.0}};
  std::printf("device %d: %d SMs, max SM clock %.0f MHz\n", dev, sms, clk_khz / 1e3);
  for (const Mix &m : mixes) {
    float best = 1e30f;
    for (int rep = 0; rep < 6; ++rep) {
      cudaEventRecord(t0);
      m.fn<<<blocks, threads>>>(out, 12345u + rep);
      cudaEventRecord(t1);
      if (!ok(cudaEventSynchronize(t1), m.name)) return 1;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, t0, t1);
      if (rep > 0 && ms < best) best = ms;  // first run warms up
    }
    const double ops = static_cast<double>(blocks) * threads * NITER * UNROLL * NCHAIN *
                       m.ops_per_step;
    const double per_s = ops / (best * 1e-3);
    const double per_clk_sm = per_s / (static_cast<double>(clk_khz) * 1e3) / sms;
    std::printf("%-22s %8.3f ms  %7.2f Tops/s  %6.1f ops/clk/SM at the max clock\n", m.name,
                best, per_s / 1e12, per_clk_sm);
  }
  cudaFree(out);
  return ok(cudaGetLastError(), "launch") ? 0 : 1;
}
