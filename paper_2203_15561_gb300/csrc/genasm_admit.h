// Device side of the server's admission: one launch packs every admitted
// request's ASCII and one scatters every admitted pair's slot metadata,
// instead of a launch and six copies per request.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "genasm_internal.h"

namespace ga {

// Segment q: segs[q].bytes ASCII bytes (a multiple of 4, 4-aligned) at
// ascii + src, packed to out + dst (one byte per four bases).
struct PackSegment {
  uint64_t src, dst, bytes;
};

// One admitted pair: its slot and the per-slot values the step kernel reads
// (offsets into the packed-sequence and CIGAR arenas, lengths, capacity).
struct SlotRecord {
  uint64_t read_off, ref_off, cigar_off;
  uint32_t slot, read_len, ref_len, cigar_cap;
};

// max_bytes: the largest segment.
cudaError_t launch_pack_segments(const uint8_t* ascii, const PackSegment* segs, uint32_t n_segs,
                                 uint64_t max_bytes, uint8_t* out, cudaStream_t s);

// Writes each record's values at its slot and zeroes the slot's window state.
cudaError_t launch_scatter_slots(const SlotRecord* recs, uint32_t n, uint64_t* read_off,
                                 uint64_t* ref_off, uint64_t* cigar_off, uint32_t* read_len,
                                 uint32_t* ref_len, uint32_t* cigar_cap, SlotState* state,
                                 cudaStream_t s);

}  // namespace ga
