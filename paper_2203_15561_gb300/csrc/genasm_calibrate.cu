// Roofline denominators for the integer-bound distance calculation, and the
// library's launch counter.
//
// The DC is plain 32-bit integer logic: per 64-bit DP cell, two funnel shifts
// (the <<1 of the new entry, reused by the neighbouring cells) and four
// 3-input logic ops ((a|b)&c and a&b&c on each 32-bit half). No datasheet
// figure is assumed for sm_103a: these microbenchmarks measure the issue rate
// of exactly those instructions (inline PTX lop3.b32 / shf.l.wrap.b32, many
// independent chains per thread, full occupancy on every SM). A second
// microbenchmark measures the shared-memory bandwidth the table stores and
// traceback reads draw on (16-byte accesses, no bank conflicts).
#include <atomic>
#include <cstdint>

#include <cuda_runtime.h>

#include "genasm_internal.h"

namespace ga {

namespace {
std::atomic<uint64_t> g_launches{0};
}

uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void uncount_launches(uint64_t n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }

__device__ __forceinline__ uint32_t lop3_xor(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t lop3_orand(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;  // (a | b) & c
  asm("lop3.b32 %0, %1, %2, %3, 0xE0;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t lop3_and3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;  // a & b & c
  asm("lop3.b32 %0, %1, %2, %3, 0x80;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t shf_l(uint32_t lo, uint32_t hi) {
  uint32_t d;  // upper word of (hi:lo) << 1
  asm("shf.l.wrap.b32 %0, %1, %2, 1;" : "=r"(d) : "r"(lo), "r"(hi));
  return d;
}

constexpr int kChains = 8;
constexpr int kUnroll = 16;

// MODE 0: LOP3 only; 1: SHF only; 2: DC cell mix (2 SHF + 4 LOP3 per cell).
template <int MODE>
__global__ void __launch_bounds__(256) int_peak_kernel(uint32_t* out, int iters, uint32_t seed) {
  uint32_t a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = (threadIdx.x + 977u * c) ^ seed;
  const uint32_t k1 = seed * 2654435761u, k2 = seed ^ 0x9e3779b9u;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      if (MODE == 0) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = lop3_xor(a[c], k1, k2);
      } else if (MODE == 1) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = shf_l(k1, a[c]);
      } else {
        // kChains/2 cells, each a (lo, hi) pair: 2 SHF + 4 LOP3.
#pragma unroll
        for (int c = 0; c < kChains; c += 2) {
          const uint32_t lo = a[c], hi = a[c + 1];
          const uint32_t hs = shf_l(lo, hi);
          const uint32_t ls = shf_l(k2, lo);
          a[c] = lop3_and3(lop3_orand(ls, k1, lo), k2, hi);
          a[c + 1] = lop3_and3(lop3_orand(hs, k1, hi), k2, lo);
        }
      }
    }
  }
  uint32_t x = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) x ^= a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = x;
}

template <int MODE>
static cudaError_t time_mode(uint32_t* buf, int blocks, int iters, cudaStream_t s, double* ops_s) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  int_peak_kernel<MODE><<<blocks, 256, 0, s>>>(buf, iters / 8, 1u);  // warm-up
  cudaEventRecord(e0, s);
  int_peak_kernel<MODE><<<blocks, 256, 0, s>>>(buf, iters, 12345u);
  cudaEventRecord(e1, s);
  count_launches(2);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  const double per_iter = MODE == 2 ? (kChains / 2) * 6.0 * kUnroll : kChains * 1.0 * kUnroll;
  *ops_s = static_cast<double>(blocks) * 256.0 * iters * per_iter / (ms * 1e-3);
  return cudaSuccess;
}

cudaError_t measure_int_peak(double out[3], cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int blocks = sms * 8;  // 2048 threads per SM
  uint32_t* buf = nullptr;
  if ((e = cudaMalloc(&buf, sizeof(uint32_t) * blocks * 256)) != cudaSuccess) return e;
  const int iters = 4096;
  e = time_mode<0>(buf, blocks, iters, s, &out[0]);
  if (e == cudaSuccess) e = time_mode<1>(buf, blocks, iters, s, &out[1]);
  if (e == cudaSuccess) e = time_mode<2>(buf, blocks, iters / 2, s, &out[2]);
  cudaFree(buf);
  return e;
}

constexpr int kSmemRows = 4;  // rows of 256 x 16 bytes per block

// MODE 0: 16-byte shared loads, 1: 16-byte shared stores. A warp's access
// covers 512 contiguous bytes (four full 128-byte wavefronts); a thread
// touches kSmemRows addresses 4 KB apart per unrolled step. The accesses are
// volatile: the addresses repeat every iteration, and plain loads of
// unchanging shared memory may be hoisted out of the loop.
template <int MODE>
__global__ void __launch_bounds__(256) smem_peak_kernel(uint32_t* out, int iters, uint32_t seed) {
  extern __shared__ __align__(16) uint4 sm[];
  const int t = threadIdx.x;
  for (int r = 0; r < kSmemRows; ++r) sm[r * 256 + t] = make_uint4(t ^ seed, r, seed, t);
  __syncthreads();
  const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(sm)) + 16u * t;
  uint32_t x = seed;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int r = 0; r < kSmemRows; ++r) {
        const uint32_t a = base + 4096u * r;
        if (MODE == 0) {
          uint32_t v0, v1, v2, v3;
          asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                       : "=r"(v0), "=r"(v1), "=r"(v2), "=r"(v3) : "r"(a));
          x ^= lop3_xor(v0, v1, v2) ^ v3;
        } else {
          asm volatile("st.volatile.shared.v4.u32 [%0], {%1, %2, %3, %4};"
                       ::"r"(a), "r"(x), "r"(x ^ 1u), "r"(x ^ 2u), "r"(x ^ 3u) : "memory");
          x += 1u;
        }
      }
    }
  }
  __syncthreads();
  out[blockIdx.x * blockDim.x + t] = x ^ sm[t].x;
}

template <int MODE>
static cudaError_t time_smem(uint32_t* buf, int blocks, int iters, cudaStream_t s, double* bytes_s) {
  constexpr size_t kBytes = sizeof(uint4) * 256 * kSmemRows;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  smem_peak_kernel<MODE><<<blocks, 256, kBytes, s>>>(buf, iters / 8, 1u);  // warm-up
  cudaEventRecord(e0, s);
  smem_peak_kernel<MODE><<<blocks, 256, kBytes, s>>>(buf, iters, 12345u);
  cudaEventRecord(e1, s);
  count_launches(2);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  *bytes_s = static_cast<double>(blocks) * 256.0 * iters * kUnroll * kSmemRows * 16.0 / (ms * 1e-3);
  return cudaSuccess;
}

cudaError_t measure_smem_peak(double out[2], cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int blocks = sms * 8;  // 2048 threads and 128 KB of shared memory per SM
  uint32_t* buf = nullptr;
  if ((e = cudaMalloc(&buf, sizeof(uint32_t) * blocks * 256)) != cudaSuccess) return e;
  const int iters = 2048;
  e = time_smem<0>(buf, blocks, iters, s, &out[0]);
  if (e == cudaSuccess) e = time_smem<1>(buf, blocks, iters, s, &out[1]);
  cudaFree(buf);
  return e;
}

}  // namespace ga
