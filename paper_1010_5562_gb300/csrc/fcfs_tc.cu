// Split-FP16 tensor-core path: the quarter-plane contraction on tcgen05 with
// the accumulator in TMEM and both operands generated on chip.
//
//   P[m, n] = sum_v A[m, v] B[n, v]  (see fcfs_simt.cu for A, B and the rows),
//   A = A_hi + A_lo, B = B_hi + B_lo (FP16, hi = rn(c), lo = rn(c - hi)),
//   P ~= A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T, accumulated in FP32 in TMEM.
//
// The dropped A_lo B_lo^T term is below 2^-22 of a term.  The corner sign s_v
// is folded into the phase (s = -1 adds T/2), so generating A costs the same
// as generating B.  CTA roles (192 threads):
//   warps 0-3   generate the A and B tiles of a 64-vertex chunk into shared
//               memory in the K-major 128-byte-swizzled layout, then drain TMEM
//               in the epilogue;
//   warp 4      allocates TMEM; lane 0 issues the tcgen05.mma (3 split
//               products x 4 k-steps per chunk) and the commits;
//   warp 5      lane 0 streams the vertex chunks (x, y, s) with 1-D TMA and
//               bulk-copies the sincos table once.
// Every mbarrier wait is bounded: on time-out the status word gets
// FCFS_ETIMEOUT and the CTA drains and exits normally.
#include "fcfs_common.cuh"

namespace fcfs {

constexpr int kBM = 128;         // tile rows (64 k values x {cos, sin})
constexpr int kCh = 64;          // vertices per chunk = one 128-byte swizzle row of FP16
constexpr int kGenWarps = 4;
constexpr int kGenThreads = kGenWarps * 32;
constexpr int kTcThreads = kGenThreads + 64;
constexpr int kVStages = 2;
constexpr int kBox = 80;         // TMA box: chunk plus up to 15 elements of alignment slack
constexpr int kVStageBytes = 896;  // x @0 (320 B), y @384 (320 B), s @768 (80 B)
constexpr uint32_t kVertexTx = kBox * 4 * 2 + kBox;

template <int BN, int STAGES>
struct TcLayout {
  static constexpr int kATile = kBM * 128;         // bytes of one FP16 A tile (hi or lo)
  static constexpr int kBTile = BN * 128;
  static constexpr int kStage = 2 * kATile + 2 * kBTile;
  static constexpr int kOps = STAGES * kStage;
};

template <int BN, int STAGES>
size_t tc_smem_bytes(int T, int full) {
  return 1024 + TcLayout<BN, STAGES>::kOps + align_up(tab_tc_bytes(T, full), 128) + kVStages * kVStageBytes + 256;
}

// (cos_hi | sin_hi << 16, cos_lo | sin_lo << 16) of phase p
template <bool FULL>
__device__ __forceinline__ uint2 tc_lookup(const uint8_t* tab, uint32_t p, uint32_t logQ) {
  if (FULL) return reinterpret_cast<const uint2*>(tab)[p];
  const uint32_t* t = reinterpret_cast<const uint32_t*>(tab);
  Quad qd = quad_split(p, logQ);
  const uint32_t c = t[qd.i1], s = t[qd.i2];
  const uint32_t sg = (qd.cneg ? 0x8000u : 0u) | (qd.sneg ? 0x80000000u : 0u);
  return make_uint2(__byte_perm(c, s, 0x5410) ^ sg, __byte_perm(c, s, 0x7632) ^ sg);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}

// Byte offset of 16-byte chunk `c` (8 vertices) of row `r` in a K-major SW128 tile.
__device__ __forceinline__ uint32_t sw128(int r, int c) {
  return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}

// Generate the rows of one row pair (cos row 2i, sin row 2i+1) for this
// thread's 8 vertices and store hi and lo.  `mul` is k (or l), `xin` the
// coordinates, `add` the phase offsets (T/2 for s = -1 on A, 0 on B).
template <bool FULL, bool MASKED>
__device__ __forceinline__ void gen_pair(const uint8_t* tab, uint32_t logQ, uint32_t mask, uint32_t mul,
                                         const uint32_t (&xin)[8], const uint32_t (&add)[8],
                                         const uint32_t (&vmask)[4], uint32_t hi_base, uint32_t lo_base,
                                         int i, int oct) {
  uint2 e[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) e[t] = tc_lookup<FULL>(tab, (mul * xin[t] + add[t]) & mask, logQ);
  uint32_t ch[4], sh[4], cl[4], sl[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    ch[j] = __byte_perm(e[2 * j].x, e[2 * j + 1].x, 0x5410);
    sh[j] = __byte_perm(e[2 * j].x, e[2 * j + 1].x, 0x7632);
    cl[j] = __byte_perm(e[2 * j].y, e[2 * j + 1].y, 0x5410);
    sl[j] = __byte_perm(e[2 * j].y, e[2 * j + 1].y, 0x7632);
    if (MASKED) {
      ch[j] &= vmask[j];
      sh[j] &= vmask[j];
      cl[j] &= vmask[j];
      sl[j] &= vmask[j];
    }
  }
  const int r0 = 2 * i, r1 = 2 * i + 1;
  st_shared_v4(hi_base + sw128(r0, oct), ch[0], ch[1], ch[2], ch[3]);
  st_shared_v4(hi_base + sw128(r1, oct), sh[0], sh[1], sh[2], sh[3]);
  st_shared_v4(lo_base + sw128(r0, oct), cl[0], cl[1], cl[2], cl[3]);
  st_shared_v4(lo_base + sw128(r1, oct), sl[0], sl[1], sl[2], sl[3]);
}

template <int BN, int STAGES, bool FULL>
__global__ void __launch_bounds__(kTcThreads, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmy,
                   const __grid_constant__ CUtensorMap tms, Plan pl, uint8_t* ws) {
  using L = TcLayout<BN, STAGES>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const size_t tb = tab_tc_bytes(pl.T, FULL);
  uint8_t* ops = sm;
  uint8_t* tab = sm + L::kOps;
  uint8_t* vst = tab + align_up(tb, 128);   // TMA destinations: 128-byte aligned
  uint64_t* bars = reinterpret_cast<uint64_t*>(vst + kVStages * kVStageBytes);
  uint64_t* ofull = bars;
  uint64_t* oempty = ofull + STAGES;
  uint64_t* vfull = oempty + STAGES;
  uint64_t* vempty = vfull + kVStages;
  uint64_t* accfull = vempty + kVStages;
  uint64_t* tabbar = accfull + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tabbar + 1);

  Status* st = reinterpret_cast<Status*>(ws + pl.off_status);
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;

  const int tile = blockIdx.x, split = blockIdx.y;
  const int tm = tile / pl.tiles_n, tn = tile % pl.tiles_n;
  const long long v0 = (long long)split * pl.split_len;
  const long long v1 = min((long long)pl.V, v0 + pl.split_len);
  const int nch = (int)((v1 - v0 + kCh - 1) / kCh);

  if (tid == kGenThreads + 32) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&ofull[i], kGenThreads);
      mbar_init(&oempty[i], 1);
    }
    for (int i = 0; i < kVStages; ++i) {
      mbar_init(&vfull[i], 1);
      mbar_init(&vempty[i], kGenThreads);
    }
    mbar_init(accfull, 1);
    mbar_init(tabbar, 1);
    fence_mbar_init();
  }
  if (warp == kGenWarps) {
    tmem_alloc(tmem_slot, BN);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == kGenWarps + 1) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      mbar_arrive_expect_tx(tabbar, (uint32_t)tb);
      bulk_load(tab, ws + pl.off_tab_tc, (uint32_t)tb, tabbar);
      int j = 0;
      for (; j < nch; ++j) {
        const int vs = j % kVStages;
        const uint32_t vph = (uint32_t)(j / kVStages) & 1u;
        if (!mbar_wait(&vempty[vs], vph ^ 1u, st, 1)) break;
        const long long cs = v0 + (long long)j * kCh;
        const int a0 = (int)(cs & ~15LL);
        uint8_t* d = vst + vs * kVStageBytes;
        mbar_arrive_expect_tx(&vfull[vs], kVertexTx);
        tma_load_1d(d, &tmx, a0, &vfull[vs]);
        tma_load_1d(d + 384, &tmy, a0, &vfull[vs]);
        tma_load_1d(d + 768, &tms, a0, &vfull[vs]);
      }
      // drain: every issued copy has landed before the CTA may exit
      for (int q = max(0, j - kVStages); q < j; ++q)
        mbar_wait(&vfull[q % kVStages], (uint32_t)(q / kVStages) & 1u, st, 2);
      mbar_wait(tabbar, 0, st, 3);
    }
  } else if (warp == kGenWarps) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16_f32(kBM, BN);
      const uint32_t ops_a = smem_u32(ops);
      for (int j = 0; j < nch; ++j) {
        const int stg = j % STAGES;
        const uint32_t ph = (uint32_t)(j / STAGES) & 1u;
        if (!mbar_wait(&ofull[stg], ph, st, 4)) break;
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
          tc_mma_f16(tmem, dah, dbh, idesc, (j | ks) != 0);
          tc_mma_f16(tmem, dah, dbl, idesc, 1);
          tc_mma_f16(tmem, dal, dbh, idesc, 1);
        }
        tc_commit(&oempty[stg]);
      }
      tc_commit(accfull);
    }
  } else {
    // ---------------- generators ----------------
    const int oct = tid & 7;     // vertex octet of the chunk
    const int rp = tid >> 3;     // first row pair (0..15)
    const uint32_t mask = (uint32_t)pl.T - 1u;
    const uint32_t half = (uint32_t)pl.T >> 1;
    const uint32_t logQ = (uint32_t)pl.logT - 2u;
    const uint32_t kA = (uint32_t)(tm * (kBM / 2) + 1);
    const uint32_t lB = (uint32_t)(tn * (BN / 2) + 1);
    const uint32_t ops_a = smem_u32(ops);
    bool ok = mbar_wait(tabbar, 0, st, 5);
    for (int j = 0; ok && j < nch; ++j) {
      const int vs = j % kVStages;
      const uint32_t vph = (uint32_t)(j / kVStages) & 1u;
      const int stg = j % STAGES;
      const uint32_t ph = (uint32_t)(j / STAGES) & 1u;
      if (!mbar_wait(&vfull[vs], vph, st, 6)) break;
      const long long cs = v0 + (long long)j * kCh;
      const int off = (int)(cs & 15LL);
      const uint8_t* d = vst + vs * kVStageBytes;
      const int32_t* xs = reinterpret_cast<const int32_t*>(d);
      const int32_t* ys = reinterpret_cast<const int32_t*>(d + 384);
      const int8_t* ss = reinterpret_cast<const int8_t*>(d + 768);
      uint32_t xa[8], ya[8], addA[8], zero[8], vmask[4];
      bool full = true;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int idx = off + oct * 8 + t;
        xa[t] = (uint32_t)xs[idx];
        ya[t] = (uint32_t)ys[idx];
        addA[t] = ss[idx] < 0 ? half : 0u;
        zero[t] = 0u;
        full = full && (cs + oct * 8 + t < v1);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bool a = cs + oct * 8 + 2 * q < v1, b = cs + oct * 8 + 2 * q + 1 < v1;
        vmask[q] = (a ? 0xFFFFu : 0u) | (b ? 0xFFFF0000u : 0u);
      }
      // The next TMA write into this stage is an async-proxy write; the
      // mbarrier release alone does not order it after these generic-proxy
      // loads, which may still be in flight.  The proxy fence does.
      fence_proxy_async_smem();
      mbar_arrive(&vempty[vs]);
      if (!mbar_wait(&oempty[stg], ph ^ 1u, st, 7)) break;
      const uint32_t ahi = ops_a + stg * L::kStage;
      const uint32_t alo = ahi + L::kATile;
      const uint32_t bhi = alo + L::kATile;
      const uint32_t blo = bhi + L::kBTile;
      if (full) {
#pragma unroll 1
        for (int t = 0; t < kBM / 2 / 16; ++t) {
          const int i = rp + 16 * t;
          gen_pair<FULL, false>(tab, logQ, mask, kA + i, xa, addA, vmask, ahi, alo, i, oct);
        }
      } else {
#pragma unroll 1
        for (int t = 0; t < kBM / 2 / 16; ++t) {
          const int i = rp + 16 * t;
          gen_pair<FULL, true>(tab, logQ, mask, kA + i, xa, addA, vmask, ahi, alo, i, oct);
        }
      }
#pragma unroll 1
      for (int t = 0; t < BN / 2 / 16; ++t) {
        const int i = rp + 16 * t;
        gen_pair<FULL, false>(tab, logQ, mask, lB + i, ya, zero, vmask, bhi, blo, i, oct);
      }
      fence_proxy_async_smem();
      mbar_arrive(&ofull[stg]);
    }
    // ---------------- epilogue: TMEM -> FP32 partials ----------------
    const bool acc_ok = mbar_wait(accfull, 0, st, 8);
    __syncwarp();   // tcgen05.ld is warp-collective: reconverge after the per-octet branches
    tc_fence_after();
    const int M2 = pl.M2;
    float* P = reinterpret_cast<float*>(ws + pl.off_part) + (size_t)split * M2 * M2;
    const int row = warp * 32 + lane;
    const int m = tm * kBM + row;
    if (acc_ok && nch > 0) {
#pragma unroll 1
      for (int cb = 0; cb < BN / 32; ++cb) {
        const int n0 = tn * BN + cb * 32;
        if (n0 >= M2) break;   // warp-uniform
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 32), r);
        tmem_wait_ld();
        if (m < M2) {
          float* dst = P + (size_t)m * M2 + n0;
          if (n0 + 32 <= M2 && (M2 & 3) == 0) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
              reinterpret_cast<float4*>(dst)[q] =
                  make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                              __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
          } else {
            for (int q = 0; q < 32; ++q)
              if (n0 + q < M2) dst[q] = __uint_as_float(r[q]);
          }
        }
      }
    } else if (m < M2) {
      for (int n = tn * BN; n < min(M2, tn * BN + BN); ++n) P[(size_t)m * M2 + n] = 0.f;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == kGenWarps) {
    __syncwarp();   // lane 0 ran the MMA loop alone; dealloc is warp-collective
    tc_fence_after();
    tmem_dealloc(tmem, BN);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <int BN, int STAGES, bool FULL>
static cudaError_t launch_tc(const Plan& pl, const VertexMaps& mp, void* ws, cudaStream_t st) {
  const size_t smem = tc_smem_bytes<BN, STAGES>(pl.T, FULL);
  auto kern = gemm_tc_kernel<BN, STAGES, FULL>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(pl.tiles_m * pl.tiles_n, pl.splits);
  kern<<<grid, kTcThreads, smem, st>>>(mp.x, mp.y, mp.s, pl, static_cast<uint8_t*>(ws));
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tc(const Plan& pl, const VertexMaps& mp, void* ws, cudaStream_t st) {
  if (pl.splits == 0) return cudaSuccess;
  if (pl.bn == 256) {
    if (pl.full) return launch_tc<256, 2, true>(pl, mp, ws, st);
    return cudaErrorInvalidValue;   // quarter table does not fit beside 2 stages of 256
  }
  if (pl.full) return launch_tc<128, 3, true>(pl, mp, ws, st);
  return launch_tc<128, 2, false>(pl, mp, ws, st);
}

size_t tc_smem_for(int bn, int T, int full) {
  if (bn == 256) return tc_smem_bytes<256, 2>(T, full);
  return full ? tc_smem_bytes<128, 3>(T, full) : tc_smem_bytes<128, 2>(T, full);
}

}  // namespace fcfs
