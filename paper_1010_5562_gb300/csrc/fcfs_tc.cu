// Split-FP16 tensor-core path: the quarter-plane contraction on tcgen05 with
// the accumulator in TMEM and both operands generated on chip.
//
//   P[m, n] = sum_v A[m, v] B[n, v]  (see fcfs_simt.cu for A, B and the rows),
//   A = A_hi + A_lo, B = B_hi + B_lo (FP16, hi = rn(a), lo = rn(a - hi)),
//   P ~= A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T, accumulated in FP32 in TMEM.
//
// The dropped A_lo B_lo^T term is below 2^-22 of a term.  Operand generation:
// each generator thread owns 8 vertices and a run of 8 consecutive
// frequencies f0..f0+7.  It reads cos/sin(2 pi f0 a / T) (the anchor) and
// cos/sin(2 pi a / T) (the step) from the FP32 table at exact integer phase
// indices and produces the run by angle addition, one complex FP32 multiply
// per frequency; every value is therefore a deterministic function of
// (frequency, coordinate), so the two corners of an edge still get identical
// (or exactly opposite) operands.  The corner sign s_v is folded into the
// anchor phase (s = -1 adds T/2).  COS (continuous cosine series): row m of
// the product holds sin(2 pi (m + 1) a / T) alone, so a run covers 16
// consecutive frequencies: the thread advances by two frequencies per row pair
// (a step read at phase 2a) and takes the odd one's sine from one more
// rotation.  CTA roles:
//   generator warps  write the hi and lo tiles of a 64-vertex chunk into shared
//                    memory (K-major, 128-byte swizzle); warps 0-3 then drain
//                    TMEM in the epilogue;
//   MMA warp         allocates TMEM; lane 0 issues the tcgen05.mma (3 split
//                    products x 4 k-steps per chunk; hi*hi into one FP32
//                    accumulator, the two correction products into a second)
//                    and the commits;
//   TMA warp         lane 0 streams the vertex chunks (x, y, s) with 1-D TMA
//                    and bulk-copies the sincos table once.
// Every mbarrier wait is bounded: on time-out the status word gets
// FCFS_ETIMEOUT and the CTA drains and exits normally.
#include <cstdlib>

#include "fcfs_epilogue.cuh"

namespace fcfs {

constexpr int kBM = 128;         // tile rows (64 k values x {cos, sin})
constexpr int kCh = 64;          // vertices per chunk = one 128-byte swizzle row of FP16
constexpr int kRun = 8;          // consecutive frequencies generated by one thread

// BN: output tile columns.  PAIR: the tile is computed by a CTA pair (2-SM
// MMA, M = 256): each CTA holds 128 A rows and BN/2 B rows per stage.
template <int BN, int STAGES, bool PAIR = false>
struct TcLayout {
  static constexpr int kBRows = PAIR ? BN / 2 : BN;   // B rows in this CTA's shared memory
  static constexpr int kATile = kBM * 128;             // bytes of one FP16 A tile (hi or lo)
  static constexpr int kBTile = kBRows * 128;
  static constexpr int kStage = 2 * kATile + 2 * kBTile;
  static constexpr int kOps = STAGES * kStage;
  // one generator thread per (vertex octet, run of kRun row pairs); groups of
  // such threads take chunks in turn.  A pair's half tiles are smaller: one
  // group of four warps per stage (a group owns its stage, so a stage barrier
  // is never waited on two phases ahead)
  static constexpr int kGroups = PAIR ? STAGES : 2;
  static constexpr int kRunsA = kBM / 2 / kRun;
  static constexpr int kGroupThreads = (kBM / 2 + kBRows / 2) / kRun * 8;
  static constexpr int kGenThreads = kGroups * kGroupThreads;
  static constexpr int kGenWarps = kGenThreads / 32;
  static constexpr int kThreads = kGenThreads + 64;
};

template <int BN, int STAGES, bool PAIR = false>
size_t tc_smem_bytes(int T, int full) {
  return 1024 + TcLayout<BN, STAGES, PAIR>::kOps + align_up(tab_f32_bytes(T, full), 128) + 256;
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}

__device__ __forceinline__ void ld_shared_v4(uint32_t addr, uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d) {
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(a), "=r"(b), "=r"(c), "=r"(d) : "r"(addr) : "memory");
}

// Byte offset of 16-byte chunk `c` (8 vertices) of row `r` in a K-major SW128 tile.
__device__ __forceinline__ uint32_t sw128(int r, int c) {
  return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}

__device__ __forceinline__ uint32_t h2_bits(__half2 h) {
  uint32_t u;
  memcpy(&u, &h, 4);
  return u;
}

// hi = rn_fp16(v), lo = rn_fp16(v - hi) for two neighbouring vertices (v0 in the low half)
__device__ __forceinline__ void split2(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(v0, v1);
  const float2 hf = __half22float2(h);
  hi = h2_bits(h);
  lo = h2_bits(__floats2half2_rn(v0 - hf.x, v1 - hf.y));
}

template <int BN, int STAGES, bool FULL, bool PAIR, bool COS = false>
__global__ void __launch_bounds__(TcLayout<BN, STAGES, PAIR>::kThreads, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmp, Plan pl, uint8_t* ws) {
  using L = TcLayout<BN, STAGES, PAIR>;
  constexpr int GT = L::kGenThreads;
  constexpr int GW = L::kGenWarps;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const size_t tb = tab_f32_bytes(pl.T, FULL);
  uint8_t* ops = sm;
  float* tab = reinterpret_cast<float*>(sm + L::kOps);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L::kOps + align_up(tb, 128));
  uint64_t* ofull = bars;
  uint64_t* oempty = ofull + STAGES;
  uint64_t* accfull = oempty + STAGES;
  uint64_t* tabbar = accfull + 1;
  uint64_t* tailbar = tabbar + 1;   // fused tail: bins and fixed table, then staged partials
  uint64_t* recvbar = tailbar + 2;  // cluster pair: the peer's half tile has landed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(recvbar + 1);

  Status* st = reinterpret_cast<Status*>(ws + pl.off_status);
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;

  // launched behind the prep kernel (or, in a batch, the unit-list kernel):
  // the unit list is read right away; a single clip's prologue below touches
  // no memory those kernels write, so it overlaps them
  if (pl.batch) griddep_wait();
  Unit U = unit_of_block(pl, ws, kBM, BN);
  if (!U.live) return;   // unit slots beyond the batch's count: nothing allocated yet
  // pair rank (0 issues the MMAs) and, for a pair, the 128-row half it holds:
  // blockIdx.x = 2 (pair tile) + rank, pair tile = (row pair tm/2, column tile tn)
  const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
  if (PAIR && !pl.batch) {   // a batch unit already names its pair tile (unit_of_block)
    const int ptile = blockIdx.x >> 1;
    U.tm = 2 * (ptile / pl.tiles_n) + (int)rank;
    U.tn = ptile % pl.tiles_n;
    U.P = reinterpret_cast<float*>(ws + pl.off_part) + (size_t)blockIdx.y * pl.M2 * pl.M2 +
          (size_t)U.tm * kBM * pl.M2 + (size_t)U.tn * BN;
  }
  const int tm = U.tm, tn = U.tn;
  const long long v0 = U.v0, v1 = U.v1;
  const int nch = (int)((v1 - v0 + kCh - 1) / kCh);

  if (tid == GT + 32) {
    for (int i = 0; i < STAGES; ++i) {
      // one group fills a chunk; a pair's rank-0 barrier counts both CTAs' groups
      mbar_init(&ofull[i], PAIR ? 2 * L::kGroupThreads : L::kGroupThreads);
      mbar_init(&oempty[i], 1);
    }
    mbar_init(accfull, 1);
    mbar_init(tabbar, 1);
    mbar_init(&tailbar[0], 1);
    mbar_init(&tailbar[1], 1);
    mbar_init(recvbar, 1);
    fence_mbar_init();
  }
  if (warp == GW + 1 && lane == 0 && pl.fused) prefetch_tensormap(&tmp);
  if (warp == GW) {
    if (PAIR) {   // collective with the peer's MMA warp
      tmem_alloc_pair(tmem_slot, 2 * BN);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(tmem_slot, 2 * BN);   // D1 (hi*hi) and D2 (hi*lo + lo*hi)
      tmem_relinquish();
    }
  }
  tc_fence_before();
  __syncthreads();
  // a pair's barriers are signalled from both CTAs: both must be initialised
  if (PAIR) cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // tables, bins and counters are written by the prep kernel
  if (!pl.batch) griddep_wait();

  if (warp == GW + 1) {
    // ---------------- table copy and corner binning ----------------
    if (lane == 0) {
      mbar_arrive_expect_tx(tabbar, (uint32_t)tb);
      bulk_load(tab, ws + pl.off_tab_f32, (uint32_t)tb, tabbar);
      // the fused tail reads the fixed-point table after the main loop: have it in L2 by then
      if (pl.fused) bulk_prefetch_l2(ws + pl.off_tab_fix, (uint32_t)tab_fix_bytes(pl.T, 0));
    }
    if (pl.bin_in_gemm) {
      // every corner is binned once, spread over the tiles: the CTA of tile t
      // bins the chunks j = t mod (tiles) of its vertex range (Steps 2-3)
      const int ntiles = pl.tiles_m * pl.tiles_n, tile = tm * pl.tiles_n + tn;
      for (int j = tile; j < nch; j += ntiles)
        for (int t = lane; t < kCh; t += 32) {
          const long long v = v0 + (long long)j * kCh + t;
          if (v < v1) bin_corner(pl, ws, U.clip, __ldg(pl.vx + v), __ldg(pl.vy + v), (int)__ldg(pl.vsg + v));
        }
    }
    if (lane == 0) mbar_wait(tabbar, 0, st, 3);   // the copy has landed before the CTA may exit
  } else if (warp == GW) {
    // ---------------- MMA issuer ----------------
    if (lane == 0 && rank == 0) {
      constexpr uint32_t idesc = idesc_f16_f32(PAIR ? 2 * kBM : kBM, BN);
      const uint32_t ops_a = smem_u32(ops);
      for (int j = 0; j < nch; ++j) {
        const int stg = j % STAGES;
        const uint32_t ph = (uint32_t)(j / STAGES) & 1u;
        if (!(PAIR ? mbar_wait_cluster(&ofull[stg], ph, st, 4) : mbar_wait(&ofull[stg], ph, st, 4))) break;
        tc_fence_after();
        const uint32_t ahi = ops_a + stg * L::kStage;
        const uint32_t alo = ahi + L::kATile;
        const uint32_t bhi = alo + L::kATile;
        const uint32_t blo = bhi + L::kBTile;
#pragma unroll
        for (int ks = 0; ks < kCh / 16; ++ks) {
          const uint32_t o = ks * 32;   // 16 FP16 = 32 bytes along K inside the swizzle row
          const uint64_t dah = sdesc_sw128(ahi + o), dal = sdesc_sw128(alo + o);
          const uint64_t dbh = sdesc_sw128(bhi + o), dbl = sdesc_sw128(blo + o);
          // the large hi*hi products and the small correction products go to
          // separate accumulators: each rounded add into D1 carries one 16-vertex
          // dot product instead of three, and D2 stays 2^-11 smaller
          if (PAIR) {
            tc_mma_f16_pair(tmem, dah, dbh, idesc, (j | ks) != 0);
            tc_mma_f16_pair(tmem + BN, dah, dbl, idesc, (j | ks) != 0);
            tc_mma_f16_pair(tmem + BN, dal, dbh, idesc, 1);
          } else {
            tc_mma_f16(tmem, dah, dbh, idesc, (j | ks) != 0);
            tc_mma_f16(tmem + BN, dah, dbl, idesc, (j | ks) != 0);
            tc_mma_f16(tmem + BN, dal, dbh, idesc, 1);
          }
        }
        if (PAIR) tc_commit_pair(&oempty[stg]); else tc_commit(&oempty[stg]);
      }
      if (PAIR) tc_commit_pair(accfull); else tc_commit(accfull);
    }
  } else {
    // ---------------- generators ----------------
    // group g takes chunks j = g, g + kGroups, ...; within a group, unit =
    // (vertex octet, run of kRun row pairs); runs [0, kRunsA) are A's
    // (warp-uniform: 4 runs per warp), the others B's
    const int group = tid / L::kGroupThreads;
    const int gtid = tid % L::kGroupThreads;
    const int oct = gtid & 7;
    const int run = gtid >> 3;
    const bool isA = run < L::kRunsA;
    const int i0 = kRun * (isA ? run : run - L::kRunsA);       // first row pair in the tile
    // first frequency of the run: A rows of tile row tm; B rows of column tile
    // tn (a pair's rank r holds B rows [BN/2 r, BN/2 r + BN/2))
    const uint32_t fp = isA ? (uint32_t)(tm * (kBM / 2) + 1 + i0)
                            : (uint32_t)(tn * (BN / 2) + (int)rank * (L::kBRows / 2) + 1 + i0);
    // COS: row pair p of the tile holds frequencies 2p + 1 and 2p + 2
    const uint32_t f0 = COS ? 2u * fp - 1u : fp;
    const uint32_t mask = (uint32_t)pl.T - 1u;
    const uint32_t half = (uint32_t)pl.T >> 1;
    const uint32_t logQ = (uint32_t)pl.logT - 2u;
    const uint32_t ops_a = smem_u32(ops);
    // this thread's 8 vertices of a chunk: coordinates (x for A rows, y for B
    // rows) and, for A, the corner signs, read through the read-only cache one
    // group turn ahead of use; zero past the end of the vertex range
    const int32_t* cptr = isA ? pl.vx : pl.vy;
    auto fetch = [&](int jj, uint32_t (&c)[8], uint32_t& s0, uint32_t& s1) {
      const long long first = v0 + (long long)jj * kCh + oct * 8;
      if (first + 8 <= v1 && (first & 3) == 0) {
        const int4 q0 = __ldg(reinterpret_cast<const int4*>(cptr + first));
        const int4 q1 = __ldg(reinterpret_cast<const int4*>(cptr + first) + 1);
        c[0] = (uint32_t)q0.x; c[1] = (uint32_t)q0.y; c[2] = (uint32_t)q0.z; c[3] = (uint32_t)q0.w;
        c[4] = (uint32_t)q1.x; c[5] = (uint32_t)q1.y; c[6] = (uint32_t)q1.z; c[7] = (uint32_t)q1.w;
      } else {
#pragma unroll
        for (int t = 0; t < 8; ++t) c[t] = first + t < v1 ? (uint32_t)__ldg(cptr + first + t) : 0u;
      }
      s0 = s1 = 0u;
      if (isA) {
        if (first + 8 <= v1 && (first & 7) == 0) {
          const uint2 w = __ldg(reinterpret_cast<const uint2*>(pl.vsg + first));
          s0 = w.x;
          s1 = w.y;
        } else {
#pragma unroll
          for (int t = 0; t < 8; ++t)
            if (first + t < v1) {
              const uint32_t byte = (uint32_t)(uint8_t)__ldg(pl.vsg + first + t) << (8 * (t & 3));
              if (t < 4) s0 |= byte; else s1 |= byte;
            }
        }
      }
    };
    uint32_t cc[8], cs0 = 0u, cs1 = 0u, nc8[8], ns0 = 0u, ns1 = 0u;
    if (group < nch) fetch(group, cc, cs0, cs1);
    // swizzled byte offset of this thread's 16-byte chunk in row r: (oct ^ (r & 7)) << 4;
    // rows 2(i0 + r) have r & 7 = 2r & 7 because i0 is a multiple of 8
    uint32_t xo[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) xo[c] = (uint32_t)((oct ^ c) << 4);
    bool ok = mbar_wait(tabbar, 0, st, 5);
    for (int j = group; ok && j < nch; j += L::kGroups) {
      const int stg = j % STAGES;
      const uint32_t ph = (uint32_t)(j / STAGES) & 1u;
      if (j + L::kGroups < nch) fetch(j + L::kGroups, nc8, ns0, ns1);
      const long long cs = v0 + (long long)j * kCh;
      uint32_t a[8], add[8], vmask[4];
      const long long first = cs + oct * 8;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        a[t] = cc[t];
        add[t] = (((t < 4 ? cs0 : cs1) >> (8 * (t & 3))) & 0x80u) ? half : 0u;   // s = -1: phase + T/2
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bool lo_ok = first + 2 * q < v1, hi_ok = first + 2 * q + 1 < v1;
        vmask[q] = (lo_ok ? 0xFFFFu : 0u) | (hi_ok ? 0xFFFF0000u : 0u);
      }
      const bool masked = isA && (first + 8 > v1);
      // anchors and steps from the table, before waiting for the stage
      float c[8], sn[8], wc[8], wsn[8], wc2[8], ws2[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const float2 an = f32_lookup<FULL>(tab, (f0 * a[t] + add[t]) & mask, logQ);
        const float2 w = f32_lookup<FULL>(tab, a[t] & mask, logQ);
        c[t] = an.x;
        sn[t] = an.y;
        wc[t] = w.x;
        wsn[t] = w.y;
        if (COS) {
          const float2 w2 = f32_lookup<FULL>(tab, (2u * a[t]) & mask, logQ);
          wc2[t] = w2.x;
          ws2[t] = w2.y;
        }
      }
      if (!mbar_wait(&oempty[stg], ph ^ 1u, st, 7)) break;
      const uint32_t tile_hi = ops_a + stg * L::kStage + (isA ? 0u : 2u * L::kATile) + 256u * (uint32_t)i0;
      const uint32_t lo_delta = isA ? (uint32_t)L::kATile : (uint32_t)L::kBTile;
#pragma unroll
      for (int r = 0; r < kRun; ++r) {
        if (r) {
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const float uc = COS ? wc2[t] : wc[t], us = COS ? ws2[t] : wsn[t];
            const float nc = fmaf(c[t], uc, -(sn[t] * us));
            const float ns = fmaf(sn[t], uc, c[t] * us);
            c[t] = nc;
            sn[t] = ns;
          }
        }
        uint32_t ch[4], cl[4], sh[4], sl[4];
        if (COS) {
          // rows 2(i0 + r) and 2(i0 + r) + 1: the sines of frequencies f and f + 1
          float s1[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) s1[t] = fmaf(sn[t], wc[t], c[t] * wsn[t]);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            split2(sn[2 * q], sn[2 * q + 1], ch[q], cl[q]);
            split2(s1[2 * q], s1[2 * q + 1], sh[q], sl[q]);
          }
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            split2(c[2 * q], c[2 * q + 1], ch[q], cl[q]);
            split2(sn[2 * q], sn[2 * q + 1], sh[q], sl[q]);
          }
        }
        if (masked) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            ch[q] &= vmask[q];
            cl[q] &= vmask[q];
            sh[q] &= vmask[q];
            sl[q] &= vmask[q];
          }
        }
        // cos row 2(i0 + r) and sin row 2(i0 + r) + 1 of the hi and lo tiles (COS: both sines)
        const uint32_t rc = tile_hi + 256u * r + xo[(2 * r) & 7];
        const uint32_t rs = tile_hi + 256u * r + 128u + xo[(2 * r + 1) & 7];
        st_shared_v4(rc, ch[0], ch[1], ch[2], ch[3]);
        st_shared_v4(rs, sh[0], sh[1], sh[2], sh[3]);
        st_shared_v4(rc + lo_delta, cl[0], cl[1], cl[2], cl[3]);
        st_shared_v4(rs + lo_delta, sl[0], sl[1], sl[2], sl[3]);
      }
      fence_proxy_async_smem();
      if (PAIR) mbar_arrive_cluster(&ofull[stg], 0); else mbar_arrive(&ofull[stg]);
#pragma unroll
      for (int t = 0; t < 8; ++t) cc[t] = nc8[t];
      cs0 = ns0;
      cs1 = ns1;
    }
    // ---------------- epilogue: TMEM -> FP32 partials (generator warps 0-7) ----------------
    // Warp w drains TMEM lane quadrant w mod 4 (tile rows 32 (w mod 4) ..) and
    // every other 32-column block.  A 32 x 32 block goes through a padded
    // shared-memory transpose (row stride 36 floats: the row-per-lane 16-byte
    // writes and the 4-rows-per-instruction reads are both conflict-free), so
    // each 16-byte global store instruction covers four whole 128-byte rows
    // instead of 32 scattered 16-byte pieces.  The operand stages are free:
    // the last MMA has completed.
    constexpr int kEpiWarps = GW < 8 ? GW : 8;
    if (warp < kEpiWarps) {
      const bool acc_ok = __all_sync(0xffffffffu, mbar_wait(accfull, 0, st, 8) ? 1 : 0) != 0;
      tc_fence_after();
      const int M2 = pl.M2;
      const int row0 = (warp & 3) * 32;
      const bool split_pair = !COS && pl.fused && pl.cluster == 2;
      const uint32_t tr = smem_u32(ops) + (uint32_t)warp * (32u * 36u * 4u);
#pragma unroll 1
      for (int cb = warp >> 2; cb < BN / 32; cb += kEpiWarps / 4) {
        const int n0 = tn * BN + cb * 32;
        if (n0 >= M2) break;   // warp-uniform
        uint32_t r[32];
        if (acc_ok && nch > 0) {
          uint32_t r2[32];
          tmem_ld32(tmem + ((uint32_t)row0 << 16) + (uint32_t)(cb * 32), r);
          tmem_ld32(tmem + ((uint32_t)row0 << 16) + (uint32_t)(BN + cb * 32), r2);
          tmem_wait_ld();
#pragma unroll
          for (int q = 0; q < 32; ++q) r[q] = __float_as_uint(__uint_as_float(r[q]) + __uint_as_float(r2[q]));
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) r[q] = 0u;
        }
        const int row = row0 + lane;
        if (split_pair) {
          // tile row `row` in shared memory, 16-byte chunks XOR-swizzled by row & 7
#pragma unroll
          for (int q = 0; q < 8; ++q)
            st_shared_v4(smem_u32(ops) + (uint32_t)row * (BN * 4) + ((uint32_t)((cb * 8 + q) ^ (row & 7)) << 4),
                         r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
          continue;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
          st_shared_v4(tr + (uint32_t)(lane * 36 + 4 * q) * 4u, r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
        __syncwarp();
        const int c4 = lane & 7;   // 16-byte column chunk of the block
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int rr = 4 * i + (lane >> 3);   // block row
          const int m = tm * kBM + row0 + rr, n = n0 + 4 * c4;
          uint32_t v0, v1, v2, v3;
          ld_shared_v4(tr + (uint32_t)(rr * 36 + 4 * c4) * 4u, v0, v1, v2, v3);
          if (m < M2 && n < M2) {
            float* dst = U.P + (size_t)(row0 + rr) * U.ld + cb * 32 + 4 * c4;
            if (n + 4 <= M2 && (U.ld & 3) == 0) {
              *reinterpret_cast<float4*>(dst) =
                  make_float4(__uint_as_float(v0), __uint_as_float(v1), __uint_as_float(v2), __uint_as_float(v3));
            } else {
              const uint32_t vv[4] = {v0, v1, v2, v3};
              for (int t = 0; t < 4 && n + t < M2; ++t) dst[t] = __uint_as_float(vv[t]);
            }
          }
        }
        __syncwarp();
      }
    }
  }

  if (!COS && pl.fused && pl.cluster == 2) {
    // Split pairs: the two CTAs of the cluster hold the same output tile for
    // splits 2g and 2g + 1.  Each sends the half of its tile that the other
    // sums (rows [64 r', 64 r' + 64) for peer rank r') with one bulk copy into
    // the peer's shared memory, adds the received half to its own in split
    // order and writes the sum as partial g: half the partial bytes in global
    // memory.  The operand stages are free: the last MMA has completed.
    constexpr uint32_t kRowBytes = BN * 4, kHalf = (kBM / 2) * kRowBytes;
    const uint32_t rank = cluster_ctarank(), peer = rank ^ 1u;
    const uint32_t tile = smem_u32(ops), recv = tile + kBM * kRowBytes;
    if (tid == 0) mbar_arrive_expect_tx(recvbar, kHalf);   // before the barrier the peer's copy waits for
    fence_proxy_async_smem();   // the tile (generic writes) before the bulk copy reads it
    __syncwarp();               // the barrier is warp-aligned: reconverge after the role branches
    cluster_sync_all();
    if (tid == 0) {
      bulk_copy_to_peer(mapa_shared(recv, peer), tile + peer * kHalf, kHalf, mapa_shared(smem_u32(recvbar), peer));
      bulk_commit();
    }
    const bool got = mbar_wait(recvbar, 0, st, 9);
    const int M2 = pl.M2;
    float* out = reinterpret_cast<float*>(ws + pl.off_part) + (size_t)(blockIdx.y >> 1) * M2 * M2;
    for (int e = tid; e < (kBM / 2) * (BN / 4) && got; e += L::kThreads) {
      const int rr = e / (BN / 4), c = e % (BN / 4);
      const int row = (int)rank * (kBM / 2) + rr;
      const uint32_t sw = (uint32_t)rr * kRowBytes + ((uint32_t)(c ^ (row & 7)) << 4);
      const float4 mine = *reinterpret_cast<const float4*>(ops + rank * kHalf + sw);
      const float4 theirs = *reinterpret_cast<const float4*>(ops + kBM * kRowBytes + sw);
      const float4 a = rank == 0 ? mine : theirs, b2 = rank == 0 ? theirs : mine;   // split 2g first
      const float4 v = make_float4(a.x + b2.x, a.y + b2.y, a.z + b2.z, a.w + b2.w);
      const int m = tm * kBM + row, n = tn * BN + 4 * c;
      if (m < M2 && n < M2) {
        float* dst = out + (size_t)m * M2 + n;
        if (n + 4 <= M2) {
          *reinterpret_cast<float4*>(dst) = v;
        } else {
          const float vv[4] = {v.x, v.y, v.z, v.w};
          for (int i = 0; i < M2 - n; ++i) dst[i] = vv[i];
        }
      }
    }
    if (tid == 0) bulk_wait_read_all();   // the outgoing copy has read the tile before anything reuses it
  }

  tc_fence_before();
  __syncthreads();
  // a pair's MMAs, commits and arrivals reach both CTAs: neither releases its
  // TMEM or leaves before both are done
  if (PAIR) {
    __syncwarp();
    cluster_sync_all();
  }
  if (warp == GW) {
    __syncwarp();   // lane 0 ran the MMA loop alone; dealloc is warp-collective
    tc_fence_after();
    if (PAIR) tmem_dealloc_pair(tmem, 2 * BN); else tmem_dealloc(tmem, 2 * BN);
  }
  // single clip, cooperative launch: split-K sum, axis lines and output here.
  // Every copy into shared memory has landed and every MMA has completed, so
  // the operand stages are free; TMEM is released before the grid barrier.
  if constexpr (!COS) {
    if (pl.fused) fused_tail(pl, ws, sm, reinterpret_cast<int*>(tmem_slot + 1), &tailbar[0], &tailbar[1], &tmp);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
// CTAs of one kernel variant that fit on the device at once, in clusters of
// C (1 or 2) along the split dimension, or in CTA pairs (cached per device).
template <int BN, int STAGES, bool FULL, bool PAIR>
static int tc_resident_ctas(size_t smem, int C) {
  constexpr int kMaxDev = 64;
  static int cache[kMaxDev][3] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev || C < 1 || C > 2) return 0;
  if (cache[dev][C]) return cache[dev][C];
  auto kern = gemm_tc_kernel<BN, STAGES, FULL, PAIR>;
  if (ensure_smem(reinterpret_cast<const void*>(kern), smem) != cudaSuccess) return 0;
  int n = 0;
  if (C == 1 && !PAIR) {
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TcLayout<BN, STAGES, PAIR>::kThreads, smem) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    n = per_sm * sms;
  } else {
    const int cx = PAIR ? 2 : 1, cy = PAIR ? 1 : C;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cx, cy);
    cfg.blockDim = dim3(TcLayout<BN, STAGES, PAIR>::kThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cx;
    at[0].val.clusterDim.y = cy;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, reinterpret_cast<const void*>(kern), &cfg) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    n = clusters * cx * cy;
  }
  cache[dev][C] = n;
  return n;
}

// Cluster size of a fused launch of this variant along the splits (2: split
// pairs, 1: none), 0 if the call cannot be fused.  CTA-pair launches use no
// split pairs.
template <int BN, int STAGES, bool FULL, bool PAIR>
static int fuse_cluster(const Plan& pl) {
  using L = TcLayout<BN, STAGES, PAIR>;
  if (pl.batch) return 0;
  const long long ctas = (long long)pl.tiles_m * pl.tiles_n * pl.splits;
  if (ctas < 1) return 0;
  // partial rows are bulk-copied in 16-byte units: rows of 2K floats need K even
  if (pl.K % 2 != 0) return 0;
  // the tail may use the operand stages and the FP32 table region (contiguous)
  const size_t avail = (size_t)L::kOps + align_up(tab_f32_bytes(pl.T, FULL), 128);
  const size_t smem = tc_smem_bytes<BN, STAGES, PAIR>(pl.T, FULL);
  for (int C : {2, 1}) {
    if (pl.splits % C != 0 || (PAIR && C > 1)) continue;
    // a split pair keeps its tile and the peer's half in the operand stages
    if (C == 2 && (size_t)kBM * BN * 4 * 3 / 2 > (size_t)L::kOps) continue;
    if (tail_smem(pl.T, pl.K, pl.splits / C, ctas, L::kThreads).total > avail) continue;
    if (ctas <= tc_resident_ctas<BN, STAGES, FULL, PAIR>(smem, C)) return C;
  }
  return 0;
}

template <int BN, int STAGES, bool FULL, bool PAIR, bool COS = false>
static cudaError_t launch_tc(const Plan& pl, const VertexMaps& mp, void* ws, cudaStream_t st) {
  const size_t smem = tc_smem_bytes<BN, STAGES, PAIR>(pl.T, FULL);
  auto kern = gemm_tc_kernel<BN, STAGES, FULL, PAIR, COS>;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  dim3 grid = pl.batch ? dim3(PAIR ? 2 * pl.splits : pl.splits, 1) : dim3(pl.tiles_m * pl.tiles_n, pl.splits);
  // The kernel may start while the previous kernel of the stream finishes
  // (programmatic stream serialisation; it waits for it in griddep_wait()).
  // The fused tail waits at a grid barrier, so every CTA must be resident:
  // a cooperative launch guarantees that (or refuses to launch).  Where the
  // runtime refuses programmatic serialisation with the other attributes,
  // the launch drops it.
  // FCFS_PDL=0 in the environment turns programmatic serialisation off (the
  // kernels' work is the same; profilers that replay launches may need it)
  static bool pdl_ok = !(getenv("FCFS_PDL") && atoi(getenv("FCFS_PDL")) == 0);
  // FCFS_COOPERATIVE=0 launches fused calls without the co-residency guarantee
  // (for profilers that cannot replay cooperative cluster launches; the grid
  // barrier's bounded wait reports FCFS_ETIMEOUT if the CTAs are not all resident)
  static const bool coop = !(getenv("FCFS_COOPERATIVE") && atoi(getenv("FCFS_COOPERATIVE")) == 0);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(TcLayout<BN, STAGES, PAIR>::kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[3];
  int na = 0;
  if (PAIR || (pl.fused && pl.cluster > 1)) {
    at[na].id = cudaLaunchAttributeClusterDimension;
    at[na].val.clusterDim.x = PAIR ? 2 : 1;
    at[na].val.clusterDim.y = PAIR ? 1 : pl.cluster;
    at[na++].val.clusterDim.z = 1;
  }
  if (pl.fused && coop) {
    at[na].id = cudaLaunchAttributeCooperative;
    at[na++].val.cooperative = 1;
  }
  if (pdl_ok) {
    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[na++].val.programmaticStreamSerializationAllowed = 1;
  }
  cfg.attrs = at;
  cfg.numAttrs = na;
  e = cudaLaunchKernelEx(&cfg, kern, mp.part, pl, static_cast<uint8_t*>(ws));
  if (e != cudaSuccess && pdl_ok) {
    cudaGetLastError();
    pdl_ok = false;
    cfg.numAttrs = na - 1;
    e = cudaLaunchKernelEx(&cfg, kern, mp.part, pl, static_cast<uint8_t*>(ws));
  }
  count_launch(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

int gemm_tc_fuse_cluster(const Plan& pl) {
  if (pl.splits == 0) return 0;
  if (pl.pair) return pl.full ? fuse_cluster<256, 3, true, true>(pl) : fuse_cluster<256, 2, false, true>(pl);
  if (pl.bn == 256) return pl.full ? fuse_cluster<256, 2, true, false>(pl) : 0;
  if (pl.full) return fuse_cluster<128, 3, true, false>(pl);
  return fuse_cluster<128, 2, false, false>(pl);
}

cudaError_t launch_gemm_tc(const Plan& pl, const VertexMaps& mp, void* ws, cudaStream_t st) {
  if (pl.splits == 0) return cudaSuccess;
  if (pl.cosine) {   // cosine series: CTA pairs only, never fused
    if (!pl.pair || pl.fused || pl.batch) return cudaErrorInvalidValue;
    return pl.full ? launch_tc<256, 3, true, true, true>(pl, mp, ws, st)
                   : launch_tc<256, 2, false, true, true>(pl, mp, ws, st);
  }
  if (pl.pair) return pl.full ? launch_tc<256, 3, true, true>(pl, mp, ws, st) : launch_tc<256, 2, false, true>(pl, mp, ws, st);
  if (pl.bn == 256) {
    if (pl.full) return launch_tc<256, 2, true, false>(pl, mp, ws, st);
    return cudaErrorInvalidValue;   // quarter table does not fit beside 2 stages of 256
  }
  if (pl.full) return launch_tc<128, 3, true, false>(pl, mp, ws, st);
  return launch_tc<128, 2, false, false>(pl, mp, ws, st);
}

size_t tc_smem_for(int bn, int T, int full) {
  if (bn == 256) return tc_smem_bytes<256, 2>(T, full);
  return full ? tc_smem_bytes<128, 3>(T, full) : tc_smem_bytes<128, 2>(T, full);
}

}  // namespace fcfs
