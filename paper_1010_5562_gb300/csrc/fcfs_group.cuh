// Grouping of corners by one integer coordinate in [0, T] (a counting sort),
// shared by the row-binned forward contraction (groups by y) and the grouped
// adjoint contraction (groups by y for gx and by x for gy).
//
// Per coordinate, one workspace region:
//   int32 count[S], start[S], cursor[S]   S = group_stride(T) >= T + 2, a multiple of 4
//   int8  e[ny_pad]                       exponent of the power-of-two scale of a
//                                         large group (ceil(log2 count) - 14, clamped
//                                         to [0, 15]; 0 for groups of <= 2^14 corners)
//   int32 perm[V]                         corner indices, group after group
// start[T + 1] is the number of grouped corners; corners whose coordinate is
// outside [0, T] are left out.  The group of a corner is its coordinate, or,
// for the adjoint's pruned FFT, the polyphase position of the coordinate
// (group_key).  The order inside a group is whatever the
// atomic cursors give: users must not depend on it.
#pragma once

#include "fcfs_common.cuh"

namespace fcfs {

__host__ __device__ inline int group_stride(int T) { return (T + 2 + 3) & ~3; }

__host__ __device__ inline size_t group_bytes(int64_t V, int T, int ny_pad) {
  return align_up(align_up((size_t)3 * group_stride(T) * 4 + (size_t)ny_pad, 16) + (size_t)(V > 0 ? V : 1) * 4, 256);
}

// Group of coordinate c in [0, T]: c itself (key_logP < 0), or its position in
// the polyphase order of a period T = P L, P = 2^key_logP: (c mod P) L + c / P,
// with c = T on the position of 0 (the periodic functions repeat there).
__host__ __device__ inline int group_key(int c, int T, int key_logP) {
  if (key_logP < 0) return c;
  const int b = c == T ? 0 : c;
  return (b & ((1 << key_logP) - 1)) * (T >> key_logP) + (b >> key_logP);
}

struct Groups {
  int *cnt, *start, *cur;
  int8_t* ey;
  int* perm;
};

__host__ __device__ inline Groups groups_at(uint8_t* base, int T, int ny_pad) {
  const int st = group_stride(T);
  Groups g;
  g.cnt = reinterpret_cast<int*>(base);
  g.start = g.cnt + st;
  g.cur = g.start + st;
  g.ey = reinterpret_cast<int8_t*>(g.cur + st);
  g.perm = reinterpret_cast<int*>(base + align_up((size_t)3 * st * 4 + (size_t)ny_pad, 16));
  return g;
}

// A batch of n clips grouped by y, clip by clip: count, start and cursor rows
// [n][S], exponents [n][ny_pad], then one perm[V] (start values are positions
// in it; clip c's corners fill [offsets[c], offsets[c + 1])).
__host__ __device__ inline size_t batch_group_bytes(int64_t V, int n, int T, int ny_pad) {
  return align_up(align_up((size_t)3 * n * group_stride(T) * 4 + (size_t)n * ny_pad, 16) + (size_t)(V > 0 ? V : 1) * 4,
                  256);
}
__host__ __device__ inline Groups groups_clip(uint8_t* base, int T, int ny_pad, int n, int c, int64_t V) {
  (void)V;
  const size_t st = group_stride(T);
  int* cnt0 = reinterpret_cast<int*>(base);
  Groups g;
  g.cnt = cnt0 + (size_t)c * st;
  g.start = cnt0 + (size_t)n * st + (size_t)c * st;
  g.cur = cnt0 + (size_t)2 * n * st + (size_t)c * st;
  g.ey = reinterpret_cast<int8_t*>(cnt0 + (size_t)3 * n * st) + (size_t)c * ny_pad;
  g.perm = reinterpret_cast<int*>(base + align_up((size_t)3 * n * st * 4 + (size_t)n * ny_pad, 16));
  return g;
}

// Group the V corners by c0 (and, with c1 != nullptr, separately by c1 into
// the next region, base + group_bytes), on group_key(c, T, key_logP): a memset
// and three kernels (count, scan, scatter) whatever the number of coordinates.
cudaError_t launch_grouping(const int32_t* c0, const int32_t* c1, int64_t V, int T, int ny_pad, uint8_t* base,
                            cudaStream_t st, int key_logP = -1);

}  // namespace fcfs
