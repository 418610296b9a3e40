// Layout of the streaming passes: the 16-byte-vector body of x is cut into chunks of
// kChunkBytes; chunk c belongs to CTA c mod grid.  The per-CTA compaction regions and the
// bound on the terms one thread sums follow from that assignment.
#pragma once

#include "common.cuh"

namespace gbs {

constexpr int kChunkBytes = 32768;
constexpr long long kChunkVecs = kChunkBytes / 16;

// Chunks of a body of nv 16-byte vectors.
__host__ __device__ __forceinline__ long long chunk_count(long long nv) {
  return (nv + kChunkVecs - 1) / kChunkVecs;
}
// First compaction slot of CTA g.  CTA g owns chunks g, g+G, g+2G, ... (nch/G of them, one
// more for g < nch%G) and CTA 0 also the scalar head and tail (< 2*vec elements), so a
// compacting pass can write at most that many elements into [start(g), start(g+1)).
// start(G) = nch * kChunkVecs * vec + 2 * vec is the size of the whole area.
__host__ __device__ __forceinline__ long long region_start(long long g, long long nch, long long G, int vec) {
  const long long q = nch / G, r = nch % G;
  return (g * q + (g < r ? g : r)) * kChunkVecs * vec + (g > 0 ? 2 * vec : 0);
}
// Most elements one thread visits in a pass: its share of every chunk of its CTA plus
// the scalar head / tail.
__host__ __device__ __forceinline__ long long per_thread_bound(long long nch, long long G, int vec) {
  return ((nch + G - 1) / G) * ((kChunkVecs + kThreads - 1) / kThreads) * vec + 2 * vec;
}

}  // namespace gbs
