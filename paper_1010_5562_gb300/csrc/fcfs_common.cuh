// Shared definitions of the FCFS CUDA library: status codes, the workspace
// plan, sincos table access and the inline-PTX wrappers (mbarrier, TMA bulk
// copies, tcgen05/TMEM) used by the sm_103a kernels.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fcfs.h"

namespace fcfs {

// ---------------------------------------------------------------------------
// Workspace plan (host and device agree on every offset)
// ---------------------------------------------------------------------------
constexpr int kFullTableMaxT = 8192;   // full-period tables up to this T, quarter-wave above
// tensor-core contractions hold 192 KiB of operand stages beside the FP32 table,
// so their full-period tables stop at T = 4096 (32 KiB)
constexpr int kTcFullTableMaxT = 4096;
constexpr int kWsAlign = 256;
// single clips from this period on take the axis lines by a pruned FFT of the bins
constexpr int kAxisFftMinT = 16384;

struct Plan {
  int64_t V;
  int32_t T, K, prec;
  int32_t logT;
  int32_t full;        // 1: full-period tables, 0: quarter-wave tables
  int32_t fixq;        // fixed-point scale 2^fixq of the axis-line table
  int32_t M2;          // 2K: rows (and columns) of the quarter-plane product
  float quad_scale;    // T^2 / (4 pi^2), rounded once from FP64 (Eq. Fkl)
  int32_t bm, bn;      // GEMM tile
  int32_t tiles_m, tiles_n;
  int32_t splits;      // vertex splits (split-K)
  int32_t chunk;       // vertices per pipeline chunk
  int64_t split_len;   // vertices per split, a multiple of chunk
  size_t off_status, off_tab_f32, off_tab_fix, off_axis, off_bins, off_hist, off_part, total;
  uint64_t tag;        // identifies the tables cached in this workspace layout
  // batch mode (several clips): the contraction kernels walk units
  // (clip, tile, vertex split) instead of (tile, split)
  int32_t pair;                // 1: the tensor-core contraction runs on CTA pairs (2-SM MMA,
                               //    256 x 256 tiles; a CTA holds 128 rows of each)
  int32_t bin_in_gemm;         // 1: the contraction kernel bins the corners for the axis lines
  int32_t fused;               // 1: the contraction kernel also runs the split-K sum, the
                               //    axis-line DFT and the output (cooperative launch)
  int32_t barrier_extra;       // test hook: the fused grid barrier waits for this many CTAs
                               //    more than exist (so its bounded wait runs out)
  int32_t cluster;             // fused: 2 when CTAs of consecutive split pairs form a cluster
                               //    and add their partial tiles in shared memory first, else 1
  const int32_t* vx;           // corner coordinates and signs (device; read by the
  const int32_t* vy;           //    tensor-core contraction)
  const int8_t* vsg;
  float2* F;                   // output block (fused only)
  long long* area_out;         // output area (fused only)
  int32_t batch;               // 0: one clip; 1: batch
  int32_t n_clips;
  int64_t unit_vertices;       // vertices per unit (a multiple of chunk)
  const int64_t* offsets;      // device, n_clips + 1
  size_t off_units;            // int32 unit_start[n_clips + 1] in the workspace
  // row-binned contraction (single clip, many more corners than y values):
  // the corners are grouped by y and the contraction runs over the T + 1 values
  // of y; the splits then cut the y range (split_len counts y values)
  int32_t hyb;
  int32_t ny_pad;              // T + 1 rounded up to the chunk (64)
  size_t off_ycnt;             // the corners grouped by y (fcfs_group.cuh)
  size_t off_h;                // FP16 [2][M2][ny_pad]: H = sum over a y group of s A, hi then lo
  // grouped forward with a pruned FFT along y instead of the contraction over y
  int32_t yfft;
  int32_t fft_logL;            // FFT length L = 2^fft_logL (T = P L)
  size_t off_poly;             // complex FP32 [K][P][L]: conj(H) in polyphase order
  size_t off_fftab;            // the FFT's tables (fft_tables_bytes; L = 4096 only)
  // continuous cosine series: T is twice the clip's period and the M2 = K rows
  // (and columns) of the contraction are sin(2 pi f a / T), f = 1..K, only
  int32_t cosine;
  // single clips of T >= 16384: the axis lines by a pruned FP64 FFT of the bins
  // (fcfs_axis_fft.cu) into the same fixed-point sums
  int32_t axfft;
  size_t off_axfft;            // complex FP64 [2][P][K] residue sums, then int64 [P] area parts
};

// Bin one corner for the axis lines (Steps 2-3): bin_x[x] += s y, bin_y[y] += s x
// (int64 integer atomics, exact and order-free).  Out-of-range corners are skipped.
__device__ __forceinline__ void bin_corner(const Plan& pl, uint8_t* ws, int clip, int xv, int yv, int sgn) {
  const int T = pl.T;
  if (xv < 0 || xv > T || yv < 0 || yv > T || (sgn != 1 && sgn != -1)) return;
  long long* b = reinterpret_cast<long long*>(ws + pl.off_bins) + (size_t)clip * 2 * (T + 1);
  atomicAdd(reinterpret_cast<unsigned long long*>(&b[xv]), (unsigned long long)((long long)sgn * yv));
  atomicAdd(reinterpret_cast<unsigned long long*>(&b[T + 1 + yv]), (unsigned long long)((long long)sgn * xv));
}

// Work of one CTA of a contraction kernel: output tile, vertex range, and
// where its FP32 partial tile goes (base and row stride).
struct Unit {
  int tm, tn;
  long long v0, v1;
  float* P;
  int ld;
  bool live;
  int clip;
};

// Single clip: blockIdx = (tile, split); batch: blockIdx.x = unit index.
__device__ inline Unit unit_of_block(const Plan& pl, uint8_t* ws, int bm, int bn) {
  Unit u;
  float* part = reinterpret_cast<float*>(ws + pl.off_part);
  if (!pl.batch) {
    const int tile = blockIdx.x, split = blockIdx.y;
    u.tm = tile / pl.tiles_n;
    u.tn = tile % pl.tiles_n;
    u.v0 = (long long)split * pl.split_len;
    u.v1 = min((long long)pl.V, u.v0 + pl.split_len);
    u.ld = pl.M2;
    u.P = part + (size_t)split * pl.M2 * pl.M2 + (size_t)u.tm * bm * pl.M2 + (size_t)u.tn * bn;
    u.live = true;
    u.clip = 0;
    return u;
  }
  // batch on CTA pairs: blockIdx.x = 2 unit + rank, the unit's tile is a
  // 256 x 256 pair tile of which rank r holds rows [128 r, 128 r + 128)
  const int* ustart = reinterpret_cast<const int*>(ws + pl.off_units);
  const int uid = pl.pair ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  u.live = uid < ustart[pl.n_clips];
  if (!u.live) return u;
  int lo = 0, hi = pl.n_clips;   // last clip c with ustart[c] <= uid
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (ustart[mid] <= uid) lo = mid; else hi = mid;
  }
  const int c = lo;
  u.clip = c;
  const long long cv0 = pl.offsets[c], cv1 = pl.offsets[c + 1];
  const int S = (int)((cv1 - cv0 + pl.unit_vertices - 1) / pl.unit_vertices);
  const int r = uid - ustart[c];
  const int tile = r / S, sp = r % S;
  u.v0 = cv0 + (long long)sp * pl.unit_vertices;
  u.v1 = min(cv1, u.v0 + pl.unit_vertices);
  u.ld = bn;
  if (pl.pair) {
    const int rank = (int)(blockIdx.x & 1u);   // the cluster is (2, 1, 1)
    u.tm = 2 * (tile / pl.tiles_n) + rank;
    u.tn = tile % pl.tiles_n;
    u.P = part + (size_t)uid * (2 * bm) * bn + (size_t)rank * bm * bn;
  } else {
    u.tm = tile / pl.tiles_n;
    u.tn = tile % pl.tiles_n;
    u.P = part + (size_t)uid * bm * bn;
  }
  return u;
}

// Workspace header: the status word of the last call, then the table tag.
constexpr size_t kTagOffset = 8;

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Table sizes in bytes
__host__ __device__ inline size_t tab_f32_bytes(int T, int full) {
  return full ? (size_t)T * 8 : align_up((size_t)(T / 4 + 1) * 4, 16);
}
// the fixed-point table is always quarter-wave (the axis kernels expand it)
__host__ __device__ inline size_t tab_fix_bytes(int T, int full) {
  (void)full;
  return align_up((size_t)(T / 4 + 1) * 4, 16);
}
// per clip: bin_x[T+1], bin_y[T+1] (int64)
__host__ __device__ inline size_t bins_bytes(int T) { return (size_t)2 * (T + 1) * 8; }

// Axis accumulators: int64 acc[4][K] then the int64 area
//   acc[0][k-1] = sum s y cos(2 pi k x / T) 2^q     acc[1] = sum s y sin(...) 2^q
//   acc[2][l-1] = sum s x cos(2 pi l y / T) 2^q     acc[3] = sum s x sin(...) 2^q
__host__ __device__ inline size_t axis_bytes(int K) { return align_up((size_t)(4 * K + 1) * 8, 256); }

// Device status word (first 4 bytes of the workspace)
struct Status {
  unsigned int code;
  unsigned int detail;
};

__device__ inline void set_status(Status* st, unsigned int code, unsigned int detail) {
  if (atomicCAS(&st->code, 0u, code) == 0u) st->detail = detail;
}

// ---------------------------------------------------------------------------
// Inline PTX: shared memory, mbarrier, TMA, tcgen05
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: gives up after ~kWaitCycles SM cycles (about a second), records
// FCFS_ETIMEOUT with the call site and returns false.
constexpr long long kWaitCycles = 2000000000LL;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, Status* st, unsigned site) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) {
      set_status(st, FCFS_ETIMEOUT, site);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 1-D tiled TMA load of `box` elements starting at element `coord`.
__device__ __forceinline__ void tma_load_1d(void* dst, const CUtensorMap* map, int32_t coord, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.1d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2}], [%3];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(coord), "r"(smem_u32(bar))
      : "memory");
}

// 3-D tiled TMA load of one box at (c0, c1, c2) (c0 innermost).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int32_t c0, int32_t c1, int32_t c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

// Fetch a tensor map (a __grid_constant__ kernel parameter) into the TMA
// unit's descriptor cache ahead of its first use.
__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while the previous kernel of the stream runs;
// griddep_wait() returns once that kernel has completed and its writes are
// visible (immediately when there is no such dependency), and
// griddep_launch_dependents() lets the next kernel start early.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Thread-block clusters: rank, peer addresses, barrier, bulk copy to a peer
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// shared::cluster address of the same shared-memory offset in CTA `rank`
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
// Every thread of every CTA of the cluster: orders shared-memory writes before
// the barrier with accesses to them (from any CTA of the cluster) after it.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Bulk copy from this CTA's shared memory to a peer's (dst and bar are
// shared::cluster addresses of the peer); 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_copy_to_peer(uint32_t dst, uint32_t src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "r"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the source reads of every committed bulk copy of this thread are done
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// Prefetch a 16-byte aligned range (size a multiple of 16) into L2.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Plain bulk copy global -> shared (16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// tcgen05 / TMEM
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16, one CTA.
__device__ __forceinline__ void tc_mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on `bar` once every tcgen05 op issued so far by this thread has completed.
// CTA-pair (2-SM) forms: the pair is ranks 0 and 1 of a cluster of two.
// Allocation and release are collective (one warp in each CTA); the MMA is
// issued by one thread of rank 0, reads A and B from both CTAs' shared memory
// at the same offsets (rank r holds A rows [128 r, 128 r + 128) and B rows
// [N/2 r, N/2 r + N/2)) and accumulates rows [128 r, ..) into rank r's TMEM.
__device__ __forceinline__ void tmem_alloc_pair(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish_pair() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_mma_f16_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                                uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// one arrive on the mbarrier at this offset in both CTAs of the pair once the
// pair's MMAs issued so far have completed
__device__ __forceinline__ void tc_commit_pair(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"((uint16_t)3)
      : "memory");
}
// arrive on the mbarrier at this offset in CTA `rank` of the cluster (release at cluster scope)
__device__ __forceinline__ void mbar_arrive_cluster(uint64_t* bar, uint32_t rank) {
  uint32_t a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_u32(bar)), "r"(rank));
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded like mbar_wait, for barriers that threads of the peer CTA arrive on
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity, Status* st, unsigned site) {
  if (mbar_try_wait_cluster(bar, parity)) return true;
  long long t0 = clock64();
  while (!mbar_try_wait_cluster(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) {
      set_status(st, FCFS_ETIMEOUT, site);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}

// Shared-memory matrix descriptor (sm_100 family): K-major operand, 128-byte
// swizzle, 8-row core-matrix groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);         // start address
  d |= (uint64_t)1 << 16;                           // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                           // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                           // SWIZZLE_128B
  return d;
}

// Instruction descriptor, kind::f16: A = B = FP16, D = FP32, both K-major.
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---------------------------------------------------------------------------
// Sincos tables.  Phase index p = (k * a) mod T is exact in integers; a table
// entry holds cos and sin of 2 pi p / T.  Full tables have T entries; quarter-
// wave tables hold cos(2 pi r / T) for r in [0, T/4] and rebuild both values by
// the quadrant symmetries.
// ---------------------------------------------------------------------------
struct Quad {
  uint32_t i1, i2;   // table indices of |cos| and |sin|
  uint32_t cneg, sneg;
};
__device__ __forceinline__ Quad quad_split(uint32_t p, uint32_t logQ) {
  const uint32_t Q = 1u << logQ;
  const uint32_t q = p >> logQ, r = p & (Q - 1u);
  Quad o;
  const bool odd = q & 1u;
  o.i1 = odd ? Q - r : r;
  o.i2 = odd ? r : Q - r;
  o.cneg = ((q + 1u) >> 1) & 1u;   // cos < 0 in quadrants 1, 2
  o.sneg = q >> 1;                  // sin < 0 in quadrants 2, 3
  return o;
}

// cos and sin of 2 pi p / T from the FP32 table
template <bool FULL>
__device__ __forceinline__ float2 f32_lookup(const float* tab, uint32_t p, uint32_t logQ) {
  if (FULL) return reinterpret_cast<const float2*>(tab)[p];
  Quad qd = quad_split(p, logQ);
  const float c = tab[qd.i1], s = tab[qd.i2];
  return make_float2(qd.cneg ? -c : c, qd.sneg ? -s : s);
}

// ---------------------------------------------------------------------------
// Host-side launch wrappers (defined in the .cu files)
// ---------------------------------------------------------------------------
// Tensor maps of a contraction launch
struct VertexMaps {
  CUtensorMap part;   // FP32 partials [part][row][col] (fused single-clip calls only)
};

cudaError_t launch_prep(const Plan& pl, void* ws, bool validate, cudaStream_t st);
cudaError_t launch_axis(const Plan& pl, const int32_t* x, const int32_t* y, const int8_t* s, void* ws,
                        bool validate, cudaStream_t st);
cudaError_t launch_reduce(const Plan& pl, void* ws, float* F, int64_t* area, bool validate, cudaStream_t st);
cudaError_t launch_gemm_simt(const Plan& pl, const int32_t* x, const int32_t* y, const int8_t* s, void* ws,
                             cudaStream_t st);
// Give kernel `fn` at least `bytes` of dynamic shared memory and the largest
// shared-memory carveout on the current device; the attributes are set once
// per kernel, device and size (setting them costs a driver call per launch).
cudaError_t ensure_smem(const void* fn, size_t bytes);

// Tensor-core adjoint (fcfs_adjoint_tc.cu): the plan's vx/vy point at the corners.
// The contraction covers the 2K frequency rows and 2K frequency columns of each
// coefficient matrix; the k = 0 row and the columns 1 and b are FP32 side terms.
constexpr int kAdjPairRows = 256;   // coefficient rows per CTA pair (MMA N)
struct AdjTcArgs {
  Plan pl;
  int nrows;        // 2K contraction rows of each matrix (k=1 cos, k=1 sin, ..., k=K sin)
  int nrows_pad;    // rows per matrix in the packed arrays (a multiple of kAdjPairRows)
  int kdim_pad;     // packed columns (2K rounded up to 64)
  int rtiles;       // row tiles of kAdjPairRows
  size_t off_rows;  // float4 [2][nrows_pad]: (row scale, column-1 term, column-b term, 0)
  size_t off_m0;    // float [2][kdim_pad + 4]: the k = 0 row over the columns, then its 1 and b terms
  size_t off_part;  // float [2][rtiles][V]: per-row-tile partial derivatives
  int grouped;      // 1: corners grouped by b, the MMA's M dimension over the T + 1 values of b
  int ny_pad;       // grouped: T + 1 rounded up to 64 (the groups' exponent array)
  size_t off_groups;  // grouped: by y (gx), then by x (gy) (fcfs_group.cuh)
};
// Pruned-FFT adjoint (fcfs_adjoint_fft.cu): V_k(b) by input-pruned FFTs along
// the grouped coordinate b, then per-corner dots.
struct AdjFftArgs {
  Plan pl;              // T, K, tables, status; vx, vy, vsg the corners
  const float2* dF;     // (2K+1)^2 cotangent
  size_t off_dft;       // the cotangent transposed (gy reads its rows)
  int logL, logP;       // T = P L, L = 2^logL >= 2K
  size_t off_z;         // complex FP32 [2][T/16][K+1][16]: V_k at polyphase positions b'
  size_t off_side;      // float4 [2][K+1]: const_k (re, im), lin_k (re, im)
  size_t off_groups;    // corners grouped by the polyphase position of y (gx), then of x (gy)
  size_t off_tabs;      // float2 tables of the FFTs and dots (adj_tables_bytes)
  int ny_pad;
  float* gx;
  float* gy;
};
size_t adj_fft_smem(int K, int logL);
size_t fft_tables_bytes(int T, int logL);
// axis lines of a single large clip by a pruned FFT of the bins
size_t axis_fft_bytes(int T, int K);
cudaError_t launch_axis_fft(const Plan& pl, void* ws, cudaStream_t st);
size_t adj_tables_bytes(int logL);
cudaError_t launch_adj_tables(const AdjFftArgs& ar, void* ws, cudaStream_t st);
cudaError_t launch_adj_fft(const AdjFftArgs& ar, void* ws, cudaStream_t st);
cudaError_t launch_adj_dot(const AdjFftArgs& ar, void* ws, cudaStream_t st);

// Launch-shape knobs of a call: a plan's (fcfs_plan_*) while one of its calls
// runs on this thread, else the process-wide test and tuning hooks.  Negative
// (or, for splits and unit chunks, zero) values defer to the hooks.
struct Knobs {
  int hybrid;        // 0 direct, 1 automatic, 2 grouped tensor-core, 3 grouped FFT
  int splits;        // vertex splits of a single-clip contraction (0: automatic)
  int pair;          // 1: CTA-pair tiles where eligible, 0: one-CTA tiles
  int unit_chunks;   // batch: pipeline chunks per unit (0: default)
};
const Knobs* current_knobs();
struct KnobScope {
  const Knobs* prev;
  explicit KnobScope(const Knobs* k);
  ~KnobScope();
};
int knob_splits();
// Row-binned (grouped) mode of the forward and adjoint calls: 0 never, 1 automatic, 2 forced
int hybrid_mode();
// the form knob itself: 0 direct / per corner, 1 automatic, 2 grouped tensor-core, 3 grouped FFT
int hybrid_knob();
// CTA pairs for 2K >= 256 on the split-FP16 path (fcfs_debug_set_pair)
bool pair_enabled();
cudaError_t launch_adj_tc(const AdjTcArgs& ar, const CUtensorMap& mhi, const CUtensorMap& mlo, void* ws,
                          cudaStream_t st);
// Row-binned contraction (fcfs_hybrid.cu): grouping, H, and the contraction
// over y into the plan's FP32 partial planes.
cudaError_t launch_hybrid(const Plan& pl, void* ws, cudaStream_t st);
// Grouped forward with the pruned FFT along y (fcfs_hybrid.cu, fcfs_fft.cu): grouping,
// H in polyphase order, the FFT kernel (off-axis block), then the axis-line output.
cudaError_t launch_grouped_fft(const Plan& pl, void* ws, float* F, cudaStream_t st);
cudaError_t launch_fft_y(const Plan& pl, void* ws, float* F, cudaStream_t st);
cudaError_t launch_axis_out(const Plan& pl, void* ws, float* F, int64_t* area, cudaStream_t st);
int fft_log_len(int T, int K);
// Workspace regions of the row-binned contraction placed from `base`; returns the end.
size_t hybrid_extra_bytes(int64_t V, int T, int M2, int ny_pad, size_t& off_ycnt, size_t& off_h, size_t base);
// 2-D FP16 tensor map (cols innermost), 128-byte swizzle, box box_cols x box_rows
bool encode_f16_2d_sw128(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint32_t box_cols,
                         uint32_t box_rows);

// 0: the call cannot be fused; else the cluster size (1 or 2) of the fused launch
int gemm_tc_fuse_cluster(const Plan& pl);
bool make_part_map(const Plan& pl, void* ws, int parts, CUtensorMap* map);
cudaError_t launch_gemm_tc(const Plan& pl, const VertexMaps& maps, void* ws, cudaStream_t st);
void count_launch(int n);

// Kernel timing (a measurement hook, off by default): while enabled, each
// instrumented stage of a call is bracketed by two events on the caller's
// stream, recorded under the stage's name (fcfs_kernel_timing_* in fcfs.h).
void kt_begin(const char* name, cudaStream_t st);
void kt_end(cudaStream_t st);
struct KtScope {
  cudaStream_t st;
  KtScope(const char* name, cudaStream_t s) : st(s) { kt_begin(name, s); }
  ~KtScope() { kt_end(st); }
};

// A second stream of the calling thread (one per device) for the stages of a
// call that do not depend on its main sequence: side_fork makes it wait for
// everything enqueued on the call's stream so far, side_join makes the call's
// stream wait for everything enqueued on it, so a call stays one event-ordered
// (and graph-capturable) sequence.  nullptr when the environment has
// FCFS_OVERLAP=0 or the stream cannot be created: the caller then runs the
// stage on its own stream.
struct SideStream {
  cudaStream_t s;
  cudaEvent_t fork, join;
};
SideStream* side_stream();
cudaError_t side_fork(SideStream* ss, cudaStream_t st);
cudaError_t side_join(SideStream* ss, cudaStream_t st);

}  // namespace fcfs
