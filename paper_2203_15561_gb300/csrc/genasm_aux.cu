// Input stage of the hot path: ASCII -> 2-bit packer.
//
// Each thread turns 16 ASCII bytes (one 16-byte load) into 4 packed bytes
// (one 4-byte store), two such chunks at a time, so both sides of the copy
// are fully coalesced; the kernel is bound by HBM bandwidth (1.25 bytes moved
// per base).
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "genasm_admit.h"
#include "genasm_internal.h"

namespace ga {

// A/a->0, C/c->1, G/g->2, T/t->3: bits 1-2 of the byte, with the G/T pair
// swapped by xoring bit 2 into bit 1. `ok` reports whether c is one of the
// eight accepted letters.
__device__ __forceinline__ uint32_t code_of(uint32_t c, bool& ok) {
  const uint32_t u = c | 0x20u;
  ok = u == 'a' || u == 'c' || u == 'g' || u == 't';
  return ok ? (((c >> 1) ^ (c >> 2)) & 3u) : 0u;
}

// 0x80 in each zero byte of v, exactly: the low 7 bits of a byte plus 0x7F
// stay below 0x100, so no carry crosses a byte.
__device__ __forceinline__ uint32_t zero_bytes(uint32_t v) {
  return ~(((v & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | v) & 0x80808080u;
}

// The four bases of a word as one byte (base q at bits 2q), a word at a time:
// code_of's bits 1-2 with G/T swapped, validity by comparing the lower-cased
// bytes with a, c, g and t; other bytes code 0 and are counted in `bad`.
__device__ __forceinline__ uint32_t pack4(uint32_t w, uint32_t& bad) {
  const uint32_t u = w | 0x20202020u;
  const uint32_t ok = zero_bytes(u ^ 0x61616161u) | zero_bytes(u ^ 0x63636363u) |
                      zero_bytes(u ^ 0x67676767u) | zero_bytes(u ^ 0x74747474u);
  bad += 4u - static_cast<uint32_t>(__popc(ok));
  const uint32_t c = ((w >> 1) ^ (w >> 2)) & ((ok >> 7) * 3u);  // 2-bit code per byte
  const uint32_t t = c | (c >> 6);
  return (t | (t >> 12)) & 0xffu;
}

__global__ void pack_kernel(const uint8_t* __restrict__ ascii, uint64_t n, uint8_t* __restrict__ out,
                            uint32_t* __restrict__ n_invalid) {
  const uint64_t chunks = n / 16;
  uint32_t bad = 0;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  // Two chunks per iteration: both 16-byte loads are in flight together.
  for (uint64_t q = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < chunks;
       q += 2 * stride) {
    const bool two = q + stride < chunks;
    const uint4 v = __ldcs(reinterpret_cast<const uint4*>(ascii) + q);
    const uint4 v2 = two ? __ldcs(reinterpret_cast<const uint4*>(ascii) + q + stride)
                         : make_uint4(0x41414141u, 0x41414141u, 0x41414141u, 0x41414141u);
    reinterpret_cast<uint32_t*>(out)[q] = pack4(v.x, bad) | (pack4(v.y, bad) << 8) |
                                          (pack4(v.z, bad) << 16) | (pack4(v.w, bad) << 24);
    uint32_t bad2 = 0;
    const uint32_t p2 = pack4(v2.x, bad2) | (pack4(v2.y, bad2) << 8) | (pack4(v2.z, bad2) << 16) |
                        (pack4(v2.w, bad2) << 24);
    if (two) {
      reinterpret_cast<uint32_t*>(out)[q + stride] = p2;
      bad += bad2;
    }
  }
  // Tail (n % 16 bytes): one thread, byte by byte.
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (uint64_t x = chunks * 16; x < n; x += 4) {
      uint32_t byte = 0;
      for (uint64_t y = x; y < x + 4 && y < n; ++y) {
        bool ok;
        byte |= code_of(ascii[y], ok) << (2 * (y - x));
        bad += ok ? 0u : 1u;
      }
      out[x / 4] = static_cast<uint8_t>(byte);
    }
  }
  if (n_invalid && bad) atomicAdd(n_invalid, bad);
}

// Any alignment: one thread per output byte.
__global__ void pack_bytes_kernel(const uint8_t* __restrict__ ascii, uint64_t n,
                                  uint8_t* __restrict__ out, uint32_t* __restrict__ n_invalid) {
  const uint64_t nb = (n + 3) / 4;
  uint32_t bad = 0;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t q = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < nb;
       q += stride) {
    uint32_t byte = 0;
    for (uint64_t y = 4 * q; y < 4 * q + 4 && y < n; ++y) {
      bool ok;
      byte |= code_of(ascii[y], ok) << (2 * (y - 4 * q));
      bad += ok ? 0u : 1u;
    }
    out[q] = static_cast<uint8_t>(byte);
  }
  if (n_invalid && bad) atomicAdd(n_invalid, bad);
}

// Many sequences at once: segment q packs segs[q].bytes ASCII bytes (a
// multiple of 4, starting 4-aligned) from ascii + segs[q].src into
// out + segs[q].dst, one output byte per four bases. Block row y handles
// segments y, y + gridDim.y, ...
__global__ void pack_segments_kernel(const uint8_t* __restrict__ ascii,
                                     const PackSegment* __restrict__ segs, uint32_t n_segs,
                                     uint8_t* __restrict__ out) {
  for (uint32_t q = blockIdx.y; q < n_segs; q += gridDim.y) {
    const PackSegment g = segs[q];
    const uint32_t* src = reinterpret_cast<const uint32_t*>(ascii + g.src);
    uint8_t* dst = out + g.dst;
    const uint64_t words = g.bytes / 4;
    uint32_t bad = 0;
    for (uint64_t w = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; w < words;
         w += static_cast<uint64_t>(gridDim.x) * blockDim.x)
      dst[w] = static_cast<uint8_t>(pack4(__ldcs(src + w), bad));
  }
}

cudaError_t launch_pack_segments(const uint8_t* ascii, const PackSegment* segs, uint32_t n_segs,
                                 uint64_t max_bytes, uint8_t* out, cudaStream_t s) {
  if (n_segs == 0) return cudaSuccess;
  const uint64_t words = max_bytes / 4;
  const uint32_t bx = static_cast<uint32_t>(std::min<uint64_t>((words + 255) / 256, 64));
  const uint32_t by = std::min<uint32_t>(n_segs, 4096);
  pack_segments_kernel<<<dim3(bx > 0 ? bx : 1, by), 256, 0, s>>>(ascii, segs, n_segs, out);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void scatter_slots_kernel(const SlotRecord* __restrict__ recs, uint32_t n,
                                     uint64_t* __restrict__ read_off, uint64_t* __restrict__ ref_off,
                                     uint64_t* __restrict__ cigar_off, uint32_t* __restrict__ read_len,
                                     uint32_t* __restrict__ ref_len, uint32_t* __restrict__ cigar_cap,
                                     SlotState* __restrict__ state) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const SlotRecord r = recs[i];
    read_off[r.slot] = r.read_off;
    ref_off[r.slot] = r.ref_off;
    cigar_off[r.slot] = r.cigar_off;
    read_len[r.slot] = r.read_len;
    ref_len[r.slot] = r.ref_len;
    cigar_cap[r.slot] = r.cigar_cap;
    state[r.slot] = SlotState{};
  }
}

cudaError_t launch_scatter_slots(const SlotRecord* recs, uint32_t n, uint64_t* read_off,
                                 uint64_t* ref_off, uint64_t* cigar_off, uint32_t* read_len,
                                 uint32_t* ref_len, uint32_t* cigar_cap, SlotState* state,
                                 cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const uint32_t blocks = std::min<uint32_t>((n + 255) / 256, 1024);
  scatter_slots_kernel<<<blocks, 256, 0, s>>>(recs, n, read_off, ref_off, cigar_off, read_len,
                                              ref_len, cigar_cap, state);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_pack(const uint8_t* ascii, uint64_t n, uint8_t* packed, uint32_t* n_invalid,
                        cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const uint64_t chunks = n / 16;
  const uint64_t want = (chunks + 255) / 256;
  const int blocks = static_cast<int>(want < 1 ? 1 : (want > 8ull * sms ? 8ull * sms : want));
  const bool aligned = (reinterpret_cast<uintptr_t>(ascii) % 16 == 0) &&
                       (reinterpret_cast<uintptr_t>(packed) % 4 == 0);
  if (aligned) {
    pack_kernel<<<blocks, 256, 0, s>>>(ascii, n, packed, n_invalid);
  } else {
    const uint64_t wb = ((n + 3) / 4 + 255) / 256;
    const int b2 = static_cast<int>(wb > 8ull * sms ? 8ull * sms : (wb < 1 ? 1 : wb));
    pack_bytes_kernel<<<b2, 256, 0, s>>>(ascii, n, packed, n_invalid);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace ga

// ---------------------------------------------------------------------------
// CIGAR compaction: gathers every pair's runs (written at fixed per-pair
// capacities by the alignment kernels) into one dense array, with the
// exclusive prefix sum of the run counts as offsets. Three passes: per-chunk
// sums, a scan of the chunk sums, then per-chunk offsets and a warp-per-pair
// copy.
// ---------------------------------------------------------------------------

namespace ga {

constexpr int kScanThreads = 1024;
constexpr int kScanChunk = kScanThreads;  // pairs per block

__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t* sh, uint64_t& total) {
  // Warp-level inclusive scan, then scan of the 32 warp totals.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = lane < (blockDim.x >> 5) ? sh[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;
  }
  __syncthreads();
  total = sh[31];
  const uint64_t before = warp > 0 ? sh[warp - 1] : 0ull;
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) chunk_sum_kernel(const uint32_t* __restrict__ n_runs,
                                                                 uint32_t n, uint64_t* __restrict__ sums) {
  __shared__ uint64_t sh[32];
  const uint32_t q = blockIdx.x * kScanChunk + threadIdx.x;
  const uint64_t v = q < n ? n_runs[q] : 0u;
  uint64_t total;
  block_exclusive_scan(v, sh, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One block: exclusive scan of the chunk sums in place, any count.
__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(uint64_t* sums, uint32_t n_chunks,
                                                                 uint64_t* grand_total) {
  __shared__ uint64_t sh[32];
  uint64_t carry = 0;
  for (uint32_t base = 0; base < n_chunks; base += kScanThreads) {
    const uint32_t q = base + threadIdx.x;
    const uint64_t v = q < n_chunks ? sums[q] : 0ull;
    uint64_t total;
    const uint64_t ex = block_exclusive_scan(v, sh, total);
    if (q < n_chunks) sums[q] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) *grand_total = carry;
}

__global__ void __launch_bounds__(kScanThreads) offsets_kernel(const uint32_t* __restrict__ n_runs,
                                                               uint32_t n, const uint64_t* __restrict__ sums,
                                                               const uint64_t* __restrict__ grand_total,
                                                               uint64_t* __restrict__ out_off) {
  __shared__ uint64_t sh[32];
  const uint32_t q = blockIdx.x * kScanChunk + threadIdx.x;
  const uint64_t v = q < n ? n_runs[q] : 0u;
  uint64_t total;
  const uint64_t ex = block_exclusive_scan(v, sh, total);
  if (q < n) out_off[q] = sums[blockIdx.x] + ex;
  if (blockIdx.x == 0 && threadIdx.x == 0) out_off[n] = *grand_total;
}

__global__ void gather_runs_kernel(const uint32_t* __restrict__ cigar, const uint64_t* __restrict__ cigar_off,
                                   const uint32_t* __restrict__ n_runs, uint32_t n,
                                   const uint64_t* __restrict__ out_off, uint64_t out_cap,
                                   uint32_t* __restrict__ out) {
  if (out_off[n] > out_cap) return;  // caller's buffer too small: copy nothing
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t p = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; p < n;
       p += warps) {
    const uint32_t* src = cigar + cigar_off[p];
    uint32_t* dst = out + out_off[p];
    const uint32_t cnt = n_runs[p];
    // Four loads in flight per lane (the copy is bound by memory latency,
    // not bandwidth, with one warp per pair).
    uint32_t x = lane;
    for (; x + 96 < cnt; x += 128) {
      const uint32_t v0 = __ldcs(src + x), v1 = __ldcs(src + x + 32);
      const uint32_t v2 = __ldcs(src + x + 64), v3 = __ldcs(src + x + 96);
      dst[x] = v0;
      dst[x + 32] = v1;
      dst[x + 64] = v2;
      dst[x + 96] = v3;
    }
    for (; x < cnt; x += 32) dst[x] = __ldcs(src + x);
  }
}

size_t compact_workspace_bytes(uint32_t n_pairs) {
  const size_t chunks = (static_cast<size_t>(n_pairs) + kScanChunk - 1) / kScanChunk;
  return 256 + sizeof(uint64_t) * (chunks + 1);
}

cudaError_t launch_compact(const uint32_t* cigar, const uint64_t* cigar_off, const uint32_t* n_runs,
                           uint32_t n, uint32_t* out, uint64_t out_cap, uint64_t* out_off, void* ws,
                           cudaStream_t s) {
  const uint32_t chunks = static_cast<uint32_t>((static_cast<uint64_t>(n) + kScanChunk - 1) / kScanChunk);
  uint64_t* grand = static_cast<uint64_t*>(ws);
  uint64_t* sums = reinterpret_cast<uint64_t*>(static_cast<char*>(ws) + 256);
  if (n == 0) {
    const cudaError_t e = cudaMemsetAsync(out_off, 0, sizeof(uint64_t), s);
    return e;
  }
  // The device query comes first, so that a failure leaves every output as
  // it was (nothing is enqueued).
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  chunk_sum_kernel<<<chunks, kScanThreads, 0, s>>>(n_runs, n, sums);
  scan_sums_kernel<<<1, kScanThreads, 0, s>>>(sums, chunks, grand);
  offsets_kernel<<<chunks, kScanThreads, 0, s>>>(n_runs, n, sums, grand, out_off);
  const uint64_t want = (static_cast<uint64_t>(n) * 32 + 255) / 256;
  const int blocks = static_cast<int>(std::max<uint64_t>(1, std::min<uint64_t>(want, 16ull * sms)));
  gather_runs_kernel<<<blocks, 256, 0, s>>>(cigar, cigar_off, n_runs, n, out_off, out_cap, out);
  count_launches(4);
  return cudaGetLastError();
}

}  // namespace ga
