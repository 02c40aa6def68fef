// cq_gen.cu -- device-side generator of the nested table's per-row columns
// (declarations and definitions of the values in include/cq_gen.h).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cq_gen.h"

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint32_t col, uint64_t i) {
  uint64_t z = (seed ^ ((uint64_t)(col & 0xFF) << 56)) + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Word j of a packed stream: the fields overlapping bits [32 j, 32 j + 32).
template <class F>
__device__ __forceinline__ uint32_t pack_word(uint64_t j, uint32_t w, uint64_t n_rows, F&& field) {
  const uint64_t b0 = j * 32;
  const uint64_t f0 = b0 / w, f1 = (b0 + 31) / w;
  uint32_t out = 0;
  for (uint64_t f = f0; f <= f1 && f < n_rows; ++f) {
    const uint64_t v = field(f);
    const int64_t sh = (int64_t)(f * w) - (int64_t)b0;   // field start relative to the word
    out |= sh >= 0 ? (uint32_t)(v << sh) : (uint32_t)(v >> -sh);
  }
  return out;
}

__global__ void hash_fields_kernel(uint32_t* words, uint64_t n_words, uint64_t n_rows, uint32_t w, uint64_t seed,
                                   uint32_t col) {
  const uint64_t mask = w == 32 ? 0xFFFFFFFFull : ((1ull << w) - 1);
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n_words;
       j += (uint64_t)gridDim.x * blockDim.x)
    words[j] = pack_word(j, w, n_rows, [&](uint64_t r) { return splitmix64(seed, col, r) & mask; });
}

__global__ void codes4_kernel(uint32_t* words, uint64_t n_words, const int64_t* ends, uint64_t n_runs,
                              uint64_t n_rows, uint64_t seed) {
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n_words;
       j += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t r0 = j * 8;   // 8 fields of 4 bits per word
    uint32_t out = 0;
    if (r0 < n_rows) {
      // run of the first row: the first run whose exclusive end exceeds it
      uint64_t lo = 0, hi = n_runs;
      while (lo < hi) {
        const uint64_t mid = (lo + hi) / 2;
        if ((uint64_t)ends[mid] > r0) hi = mid;
        else lo = mid + 1;
      }
      uint64_t run = lo;
      for (uint32_t k = 0; k < 8 && r0 + k < n_rows; ++k) {
        const uint64_t r = r0 + k;
        while (run < n_runs && (uint64_t)ends[run] <= r) ++run;
        if (run >= n_runs) break;   // ends stop short of n_rows: leave the rest 0
        const uint64_t s = run ? (uint64_t)ends[run - 1] : 0;
        const uint64_t len = (uint64_t)ends[run] - s, off = r - s;
        uint32_t code = 0;
        for (uint32_t c = 0; c < 15; ++c) code += (splitmix64(seed, 4, run * 15 + c) % len) <= off ? 1u : 0u;
        out |= code << (4 * k);
      }
    }
    words[j] = out;
  }
}

unsigned grid_for(uint64_t n) {
  const uint64_t b = (n + 255) / 256;
  return (unsigned)(b < 152ull * 64 ? (b ? b : 1) : 152ull * 64);
}

}  // namespace

extern "C" int cqgen_hash_fields(uint32_t* words, uint64_t n_words, uint64_t n_rows, uint32_t bit_width,
                                 uint64_t seed, uint32_t col, void* cuda_stream) {
  if (!words || bit_width < 1 || bit_width > 32 || n_words < (n_rows * bit_width + 31) / 32) return -1;
  hash_fields_kernel<<<grid_for(n_words), 256, 0, reinterpret_cast<cudaStream_t>(cuda_stream)>>>(
      words, n_words, n_rows, bit_width, seed, col);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

extern "C" int cqgen_nested_codes4(uint32_t* words, uint64_t n_words, const int64_t* c3_ends, uint64_t n_runs,
                                   uint64_t n_rows, uint64_t seed, void* cuda_stream) {
  if (!words || (n_rows && (!c3_ends || n_runs == 0)) || n_words < (n_rows * 4 + 31) / 32) return -1;
  codes4_kernel<<<grid_for(n_words), 256, 0, reinterpret_cast<cudaStream_t>(cuda_stream)>>>(
      words, n_words, c3_ends, n_runs, n_rows, seed);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
