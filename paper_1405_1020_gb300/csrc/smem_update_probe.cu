// smem_update_probe.cu -- cost of one histogram bin update in shared memory,
// three ways, at the headline filter's occupancy (4 CTAs of 64 threads per
// SM) and shape (4 histograms x 20 levels of 8-byte bins per thread, bins
// [level][histogram][thread]).
//
//   load-add-store : ld.shared.u64, 64-bit add, st.shared.u64 (what the
//                    filter kernels do), the four histograms' loads first;
//   red.add.u64    : one red.shared.add.u64 per update, no result returned;
//   2 x red.add.u32: the bin as two 32-bit planes ([level][histogram][thread]
//                    each), one red.shared.add.u32 per plane.
//
// Each thread draws its levels from a linear congruential sequence, so that
// a warp's lanes hit different levels as in the filter.  The result is
// shared-pipe clocks per warp-wide update (SM clock from the driver's maximum)
// and a checksum of the final bins, equal across the three forms (the deltas
// keep a carry out of the low 32 bits impossible, so the two-plane form holds
// the same sums).
//
// Build: python -c "from paper_1405_1020_gb300.csrc import build; build.build_smem_update_probe()"
// Run:   paper_1405_1020_gb300/smem_update_probe

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

namespace {

constexpr int kThreads = 64, kLevels = 20, kHists = 4, kIters = 4096;
constexpr uint32_t kBins = kLevels * kHists * kThreads;  // 8-byte bins per CTA

enum Form { kLoadStore = 0, kRed64 = 1, kRed32x2 = 2 };

__device__ __forceinline__ uint32_t shared_address(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

template <int FORM>
__global__ void __launch_bounds__(kThreads) update_kernel(unsigned long long *checksum,
                                                          uint32_t seed) {
  __shared__ __align__(16) unsigned long long bins[kBins];
  const uint32_t t = threadIdx.x;
  for (uint32_t i = t; i < kBins; i += kThreads) bins[i] = 0ull;
  __syncthreads();
  uint32_t x = seed * 747796405u + t * 2891336453u + blockIdx.x;
  const uint32_t base = shared_address(bins);
  for (int it = 0; it < kIters; ++it) {
    uint32_t addr[kHists];
    uint64_t delta[kHists];
#pragma unroll
    for (int k = 0; k < kHists; ++k) {
      x = x * 1664525u + 1013904223u;
      const uint32_t level = ((x >> 16) * kLevels) >> 16;  // 0 .. kLevels - 1
      const uint32_t slot = (level * kHists + static_cast<uint32_t>(k)) * kThreads + t;
      // a count of 1, an 8-bit value at bit 10 and another at bit 32
      delta[k] = 1ull | (static_cast<uint64_t>(x & 255u) << 10) |
                 (static_cast<uint64_t>((x >> 8) & 255u) << 32);
      addr[k] = FORM == kRed32x2 ? base + slot * 4u : base + slot * 8u;
    }
    if constexpr (FORM == kLoadStore) {
      unsigned long long v[kHists];
#pragma unroll
      for (int k = 0; k < kHists; ++k)
        asm volatile("ld.shared.u64 %0, [%1];" : "=l"(v[k]) : "r"(addr[k]));
#pragma unroll
      for (int k = 0; k < kHists; ++k)
        asm volatile("st.shared.u64 [%0], %1;" ::"r"(addr[k]), "l"(v[k] + delta[k]) : "memory");
    } else if constexpr (FORM == kRed64) {
#pragma unroll
      for (int k = 0; k < kHists; ++k)
        asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(addr[k]), "l"(delta[k]) : "memory");
    } else {
      const uint32_t high_plane = kBins * 4u;  // bytes from the low plane to the high one
#pragma unroll
      for (int k = 0; k < kHists; ++k) {
        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr[k]),
                     "r"(static_cast<uint32_t>(delta[k]))
                     : "memory");
        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr[k] + high_plane),
                     "r"(static_cast<uint32_t>(delta[k] >> 32))
                     : "memory");
      }
    }
  }
  __syncthreads();
  unsigned long long sum = 0;
  if constexpr (FORM == kRed32x2) {
    const uint32_t *plane = reinterpret_cast<const uint32_t *>(bins);
    for (uint32_t i = t; i < kBins; i += kThreads)
      sum += plane[i] + (static_cast<unsigned long long>(plane[i + kBins]) << 32);
  } else {
    for (uint32_t i = t; i < kBins; i += kThreads) sum += bins[i];
  }
  atomicAdd(checksum + blockIdx.x, sum);
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
  const int blocks = sms * 4;
  unsigned long long *sums = nullptr;
  if (!ok(cudaMalloc(&sums, sizeof(unsigned long long) * blocks * 3), "cudaMalloc")) return 1;
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  struct Variant {
    const char *name;
    void (*fn)(unsigned long long *, uint32_t);
  } forms[3] = {{"load-add-store u64", update_kernel<kLoadStore>},
                {"red.shared.add.u64", update_kernel<kRed64>},
                {"2 x red.shared.add.u32", update_kernel<kRed32x2>}};
  std::printf("device %d: %d SMs, max SM clock %.0f MHz; %d CTAs of %d threads\n", dev, sms,
              clk_khz / 1e3, blocks, kThreads);
  unsigned long long first[3] = {0, 0, 0};
  for (int f = 0; f < 3; ++f) {
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      cudaMemset(sums + f * blocks, 0, sizeof(unsigned long long) * blocks);
      cudaEventRecord(t0);
      forms[f].fn<<<blocks, kThreads>>>(sums + f * blocks, 7u);
      cudaEventRecord(t1);
      if (!ok(cudaEventSynchronize(t1), forms[f].name)) return 1;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, t0, t1);
      if (rep > 0 && ms < best) best = ms;  // the first run warms up
    }
    const double warp_updates = static_cast<double>(blocks) * kThreads / 32.0 * kIters * kHists;
    const double clocks_per_sm = best * 1e-3 * clk_khz * 1e3;
    std::printf("%-24s %8.3f ms  %6.2f SM clocks per warp-wide update\n", forms[f].name, best,
                clocks_per_sm * sms / warp_updates);
    cudaMemcpy(&first[f], sums + f * blocks, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  }
  const bool same = first[0] == first[1] && first[0] == first[2];
  std::printf("checksums %llx %llx %llx: %s\n", first[0], first[1], first[2],
              same ? "equal" : "DIFFER");
  cudaFree(sums);
  return same && ok(cudaGetLastError(), "launch") ? 0 : 1;
}
