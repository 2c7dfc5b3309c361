// Split-FP16 tensor-core adjoint: the contraction of the adjoint (see
// fcfs_adjoint.cu for the formulation) on tcgen05, in CTA pairs.
//
// For matrix m (0: gx, 1: gy) and corner v with contraction coordinate b
// (y for gx, x for gy) and epilogue coordinate a (x for gx, y for gy), the
// coefficient matrix M (rows: k = 0 | cos, sin of k for k = 1..K; columns: cos,
// sin of l for l = 1..K | 1 | b) splits into the frequency block Mf (rows and
// columns below 2K), the k = 0 row m0 and the columns 1 and b (s1, sb), so the
// partial of row tile t is
//   part[m][t][v] = sum_{r in t} A'[r, v] (sum_c Mf[r, c] B'[c, v] + s1[r] + sb[r] b)
//                 + [t = 0] (sum_c m0[c] B'[c, v] + m0_1 + m0_b b),
// with B'[., v] = (cos, sin of 2 pi l b / T)_l and A'[., v] = (cos, sin of 2 pi k a / T)_k,
// rows and columns ordered (k=1 cos, k=1 sin, ..., k=K sin).
//
// Z = Mf B' runs on the tensor cores with the corners as the MMA's M
// dimension: a CTA pair holds 256 corners (128 per CTA, TMEM lane = corner)
// against 256 rows of Mf (N; each CTA stages 128 of them), contracted over the
// columns in chunks of 64 by cta_group::2 MMAs that the pair's rank 0 issues.
// Mf is packed once per call as FP16 hi + lo with a power-of-two scale per row
// and streamed by TMA in 128-byte swizzled K-major tiles; B' is generated on
// chip from the exact integer phase l b mod T (run anchors from a two-level
// sincos table, angle addition over runs of 8 frequencies, hi = rn(v),
// lo = rn(v - hi)).  Products hi*hi go to accumulator D1, hi*lo + lo*hi to D2.
// The side terms stay FP32: the generator threads of row tile 0 accumulate the
// k = 0 row from the B' values they generate, and the epilogue adds s1 + sb b
// to each row before the per-corner dot with A'.
//
// Grouped form (many more corners than values of b): B' depends on the corner
// only through b, so the MMA's M dimension runs over the T + 1 values of b
// instead of the V corners (Z[r, b] for every b), and the epilogue takes the
// corners of the CTA's 128 values of b (grouped by b, fcfs_group.cuh): Z goes
// from TMEM to shared memory (row scale and side terms applied), then each
// thread forms the dot of one corner at a time with its A' over the tile's 256
// rows.
#include <algorithm>

#include "fcfs_common.cuh"
#include "fcfs_fft.cuh"
#include "fcfs_group.cuh"

namespace fcfs {

namespace {

constexpr int kVP = 128;                  // corners per CTA (TMEM lanes)
constexpr int kRH = kAdjPairRows / 2;     // coefficient rows staged per CTA
constexpr int kAC = 64;                   // columns per chunk = one 128-byte swizzle row of FP16
constexpr int kGen = 256;                 // generator / epilogue threads: two per corner
constexpr int kThreadsA = kGen + 64;      // + MMA warp + TMA warp
constexpr int kTile = 128 * 128;          // one 128-row FP16 tile of a chunk (hi or lo), bytes
constexpr int kStage = 4 * kTile;         // corners hi, lo (generated), coefficient rows hi, lo (TMA)
constexpr int kStages = 3;
constexpr int kOps = kStages * kStage;
constexpr int kTlMax = 512;               // two-level table entries for T <= 2^16
constexpr int kM0Cache = 2048;            // k = 0 row columns kept in shared memory (2K <= 2048)
constexpr size_t kAdjSmem = 1024 + kOps + kTlMax * 8 + kAdjPairRows * 16 + 2 * kVP * 4 + kM0Cache * 4 + 256;
// grouped epilogue: Z [256 rows][128 b] FP32 and staged corners in the operand stages
constexpr int kZBytes = kAdjPairRows * kVP * 4;
constexpr int kCornerCache = (kOps - kZBytes) / 16;
static_assert(kCornerCache >= 1024, "room for staged corners");

__device__ __forceinline__ void st_shared_v4a(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ uint32_t h2bits(__half2 h) {
  uint32_t u;
  memcpy(&u, &h, 4);
  return u;
}
__device__ __forceinline__ void split_pair(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(v0, v1);
  const float2 hf = __half22float2(h);
  hi = h2bits(h);
  lo = h2bits(__floats2half2_rn(v0 - hf.x, v1 - hf.y));
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int32_t c0, int32_t c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

template <bool GROUPED>
__global__ void __launch_bounds__(kThreadsA, 1)
    adj_tc_kernel(const __grid_constant__ CUtensorMap mhi, const __grid_constant__ CUtensorMap mlo, AdjTcArgs ar,
                  uint8_t* ws) {
  constexpr int GW = kGen / 32;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const Plan& pl = ar.pl;
  uint8_t* ops = sm;
  float2* tlt = reinterpret_cast<float2*>(sm + kOps);
  float4* rows = reinterpret_cast<float4*>(tlt + kTlMax);        // this pair's 256 row terms
  float* comb = reinterpret_cast<float*>(rows + kAdjPairRows);   // [2][kVP]: column halves of each corner
  float* m0s = comb + 2 * kVP;                                    // [kM0Cache]: the k = 0 row (row tile 0)
  uint64_t* ofull = reinterpret_cast<uint64_t*>(m0s + kM0Cache); // [kStages] rank 0: rank 1's chunk is ready
  uint64_t* tfull = ofull + kStages;                             // [kStages] this CTA's rows landed
  uint64_t* gfull = tfull + kStages;                             // [kStages] this CTA's corners are generated
  uint64_t* empty = gfull + kStages;                             // [kStages] the chunk's MMAs completed
  uint64_t* accfull = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accfull + 1);

  Status* st = reinterpret_cast<Status*>(ws + pl.off_status);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // blockIdx.x = 2 (corner pair tile) + rank; rank r holds corners [128 r, 128 r + 128)
  // of the pair tile (grouped: values of b) and coefficient rows [128 r, 128 r + 128)
  // of row tile rt
  const uint32_t rank = cluster_ctarank();
  const int rt = blockIdx.y, mat = blockIdx.z;
  const long long vbase = (long long)(blockIdx.x >> 1) * (2 * kVP) + (long long)rank * kVP;
  const int r0 = rt * kAdjPairRows;
  const int nch = ar.kdim_pad / kAC;
  // this thread's corner coordinates, loaded first so that their latency
  // overlaps the prologue (generator threads: corner tid mod 128)
  const long long v_me = vbase + (tid & (kVP - 1));
  const bool live_me = tid < kGen && (GROUPED ? v_me <= pl.T : v_me < pl.V);
  const uint32_t b_me = !live_me ? 0u : (GROUPED ? (uint32_t)v_me : (uint32_t)__ldg((mat == 0 ? pl.vy : pl.vx) + v_me));
  const uint32_t a_me = (!live_me || GROUPED) ? 0u : (uint32_t)__ldg((mat == 0 ? pl.vx : pl.vy) + v_me);

  if (tid == kGen + 32) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&ofull[i], 1);             // rank 1's forwarder (its corners and rows)
      mbar_init(&gfull[i], kGen / 32);     // this CTA's generator warps
      mbar_init(&tfull[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(accfull, 1);
    fence_mbar_init();
  }
  if (warp == GW) {   // collective with the peer's MMA warp: D1 at 0, D2 at 256
    tmem_alloc_pair(tmem_slot, 2 * kAdjPairRows);
    tmem_relinquish_pair();
  }
  const uint32_t logT = (uint32_t)pl.logT, f = (logT + 1u) / 2u, nc = 1u << (logT - f);
  const TwoLevel tl{tlt, f, (1u << f) - 1u, nc};
  if (tid < kGen) {
    const float* gt = reinterpret_cast<const float*>(ws + pl.off_tab_f32);
    const uint32_t logQ = logT - 2u;
    for (uint32_t i = tid; i < nc + (1u << f); i += kGen) {
      const uint32_t p = i < nc ? i << f : i - nc;
      tlt[i] = pl.full ? f32_lookup<true>(gt, p, logQ) : f32_lookup<false>(gt, p, logQ);
    }
    const float4* gr = reinterpret_cast<const float4*>(ws + ar.off_rows) + (size_t)mat * ar.nrows_pad + r0;
    for (int i = tid; i < kAdjPairRows; i += kGen) rows[i] = __ldg(gr + i);
    // the k = 0 row (row tile 0 only): read from shared memory by the generators
    if (rt == 0 && ar.kdim_pad <= kM0Cache) {
      const float* m0g = reinterpret_cast<const float*>(ws + ar.off_m0) + (size_t)mat * (ar.kdim_pad + 4);
      for (int i = tid; i < ar.kdim_pad; i += kGen) m0s[i] = __ldg(m0g + i);
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();   // the pair's barriers are signalled from both CTAs
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t mask = (uint32_t)pl.T - 1u;
  const int K = pl.K;

  if (warp == GW + 1) {
    // ---------------- coefficient rows (TMA) ----------------
    if (lane == 0) {
      prefetch_tensormap(&mhi);
      prefetch_tensormap(&mlo);
      const int row = mat * ar.nrows_pad + r0 + (int)rank * kRH;
      int j = 0;
      for (; j < nch; ++j) {
        const int s = j % kStages;
        const uint32_t ph = (uint32_t)(j / kStages) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, st, 40)) break;
        uint8_t* bt = ops + (size_t)s * kStage + 2 * kTile;
        mbar_arrive_expect_tx(&tfull[s], 2u * kTile);
        tma_load_2d(bt, &mhi, j * kAC, row, &tfull[s]);
        tma_load_2d(bt + kTile, &mlo, j * kAC, row, &tfull[s]);
      }
      // every issued copy has landed before the CTA may exit
      for (int q = max(0, j - kStages); q < j; ++q)
        mbar_wait(&tfull[q % kStages], (uint32_t)(q / kStages) & 1u, st, 41);
    }
  } else if (warp == GW) {
    if (lane == 0 && rank == 0) {
      // ---------------- MMA issuer (rank 0 for the pair) ----------------
      constexpr uint32_t idesc = idesc_f16_f32(2 * kVP, kAdjPairRows);
      const uint32_t ops_a = smem_u32(ops);
      for (int j = 0; j < nch; ++j) {
        const int s = j % kStages;
        const uint32_t ph = (uint32_t)(j / kStages) & 1u;
        if (!mbar_wait(&gfull[s], ph, st, 44) || !mbar_wait(&tfull[s], ph, st, 47) ||
            !mbar_wait_cluster(&ofull[s], ph, st, 43))
          break;
        tc_fence_after();
        const uint32_t ahi = ops_a + s * kStage, alo = ahi + kTile, bhi = alo + kTile, blo = bhi + kTile;
#pragma unroll
        for (int ks = 0; ks < kAC / 16; ++ks) {
          const uint32_t o = ks * 32;
          const uint64_t dah = sdesc_sw128(ahi + o), dal = sdesc_sw128(alo + o);
          const uint64_t dbh = sdesc_sw128(bhi + o), dbl = sdesc_sw128(blo + o);
          tc_mma_f16_pair(tmem, dah, dbh, idesc, (j | ks) != 0);
          tc_mma_f16_pair(tmem + kAdjPairRows, dah, dbl, idesc, (j | ks) != 0);
          tc_mma_f16_pair(tmem + kAdjPairRows, dal, dbh, idesc, 1);
        }
        tc_commit_pair(&empty[s]);
      }
      tc_commit_pair(accfull);
    } else if (lane == 0) {
      // rank 1: each chunk's corners are generated and its rows have landed
      // here -> one arrival (release at cluster scope) on rank 0's barrier, so
      // that the generator warps only arrive locally
      for (int j = 0; j < nch; ++j) {
        const int s = j % kStages;
        const uint32_t ph = (uint32_t)(j / kStages) & 1u;
        if (!mbar_wait(&gfull[s], ph, st, 42) || !mbar_wait(&tfull[s], ph, st, 48)) break;
        mbar_arrive_cluster(&ofull[s], 0);
      }
    }
  } else {
    // ---------------- generators: two threads per corner ----------------
    // Thread (corner i, half g) writes columns 32 g .. 32 g + 31 of row i of
    // each chunk: l = 32 j + 16 g + 1 .. + 16 as (cos, sin) pairs, zeros past K.
    const int cidx = tid & (kVP - 1), g = tid >> 7;
    const long long v = v_me;   // the corner, or (grouped) the value b itself
    const bool live = live_me;
    const int32_t* cbp = mat == 0 ? pl.vy : pl.vx;
    const uint32_t b = b_me;
    const float* m0 = reinterpret_cast<const float*>(ws + ar.off_m0) + (size_t)mat * (ar.kdim_pad + 4);
    const float* m0r = ar.kdim_pad <= kM0Cache ? m0s : m0;   // the shared copy when it fits
    const bool krow = rt == 0;   // row tile 0 also carries the k = 0 row
    const float2 w = tl_lookup(tl, b & mask);   // step cos, sin(2 pi b / T)
    const uint32_t ops_a = smem_u32(ops);
    float acc0 = 0.f, acc0b = 0.f;   // chains over the cos and the sin columns
    for (int j = 0; j < nch; ++j) {
      const int s = j % kStages;
      const uint32_t ph = (uint32_t)(j / kStages) & 1u;
      // warp-uniform: the warp's lanes arrive together below
      if (!__all_sync(0xffffffffu, mbar_wait(&empty[s], ph ^ 1u, st, 45) ? 1 : 0)) break;
      const uint32_t hi_row = ops_a + s * kStage + (uint32_t)cidx * 128u;
#pragma unroll
      for (int run = 0; run < 2; ++run) {
        const int q = 2 * g + run;              // run of 8 frequencies = 16 columns = two 16-byte chunks
        const int l0 = 32 * j + 8 * q + 1;
        float cv[8], sv[8];
        if (l0 + 7 <= K) {
          const float2 an = tl_lookup(tl, (uint32_t)l0 * b & mask);
          float c = an.x, sn = an.y;
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            cv[t] = c;
            sv[t] = sn;
            const float c1 = fmaf(c, w.x, -(sn * w.y)), s1 = fmaf(sn, w.x, c * w.y);
            c = c1;
            sn = s1;
          }
        } else {
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            cv[t] = sv[t] = 0.f;
            if (l0 + t <= K) {
              const float2 e = tl_lookup(tl, (uint32_t)(l0 + t) * b & mask);
              cv[t] = e.x;
              sv[t] = e.y;
            }
          }
        }
        if (!live) {
#pragma unroll
          for (int t = 0; t < 8; ++t) cv[t] = sv[t] = 0.f;
        }
        if (krow) {
          const float4* mp = reinterpret_cast<const float4*>(m0r + 2 * (l0 - 1));
          float4 m[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) m[u] = mp[u];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            acc0 = fmaf(m[u].x, cv[2 * u], acc0);
            acc0b = fmaf(m[u].y, sv[2 * u], acc0b);
            acc0 = fmaf(m[u].z, cv[2 * u + 1], acc0);
            acc0b = fmaf(m[u].w, sv[2 * u + 1], acc0b);
          }
        }
        uint32_t hv[8], lv[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) split_pair(cv[t], sv[t], hv[t], lv[t]);
        const uint32_t c0 = (uint32_t)(2 * q), c1 = c0 + 1;
        const uint32_t o0 = (c0 ^ (uint32_t)(cidx & 7)) << 4, o1 = (c1 ^ (uint32_t)(cidx & 7)) << 4;
        st_shared_v4a(hi_row + o0, hv[0], hv[1], hv[2], hv[3]);
        st_shared_v4a(hi_row + o1, hv[4], hv[5], hv[6], hv[7]);
        st_shared_v4a(hi_row + kTile + o0, lv[0], lv[1], lv[2], lv[3]);
        st_shared_v4a(hi_row + kTile + o1, lv[4], lv[5], lv[6], lv[7]);
      }
      // every lane's writes are made visible to the tensor core's proxy, then
      // one arrival per warp on this CTA's barrier
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&gfull[s]);
    }

    acc0 += acc0b;

    // ---------------- epilogue: per-corner dot with A' ----------------
    // warp w reads TMEM lanes 32 (w mod 4) .. +31 (its corners, or values of b)
    // over the columns of tile rows [128 g, 128 g + 128)
    const bool acc_ok = __all_sync(0xffffffffu, mbar_wait(accfull, 0, st, 46) ? 1 : 0) != 0;
    tc_fence_after();
    if constexpr (GROUPED) {
      // (1) Z[r, b] -> shared memory zs[f][b - b0] = (cos row 2f, sin row 2f + 1)
      // with the row scale and the side terms; the operand stages are free:
      // the last MMA has completed
      float2* zs = reinterpret_cast<float2*>(ops);
      const float fb = (float)b;
      const uint32_t lane_base = ((uint32_t)(warp & 3) * 32u) << 16;
      for (int cb = 0; cb < kRH; cb += 32) {
        const int n0 = g * kRH + cb;
        uint32_t d1[32], d2[32];
        if (acc_ok) {
          tmem_ld32(tmem + lane_base + (uint32_t)n0, d1);
          tmem_ld32(tmem + lane_base + (uint32_t)(kAdjPairRows + n0), d2);
          tmem_wait_ld();
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) d1[i] = d2[i] = 0u;
        }
#pragma unroll
        for (int i = 0; i < 32; i += 2) {
          const float4 q0 = rows[n0 + i], q1 = rows[n0 + i + 1];
          zs[((n0 + i) / 2) * kVP + cidx] =
              make_float2(fmaf(__uint_as_float(d1[i]) + __uint_as_float(d2[i]), q0.x, fmaf(q0.z, fb, q0.y)),
                          fmaf(__uint_as_float(d1[i + 1]) + __uint_as_float(d2[i + 1]), q1.x, fmaf(q1.z, fb, q1.y)));
        }
      }
      comb[g * kVP + cidx] = acc0;   // the k = 0 row's two column halves (row tile 0)
      // (2) the corners whose b falls in [b0, b0 + 128), staged in pieces
      const Groups gr = groups_at(ws + ar.off_groups + (size_t)mat * group_bytes(pl.V, pl.T, ar.ny_pad), pl.T,
                                  ar.ny_pad);
      int4* sc = reinterpret_cast<int4*>(ops + kZBytes);
      const int b0 = (int)vbase;
      const int cs = gr.start[min(b0, pl.T + 1)], ce = gr.start[min(b0 + kVP, pl.T + 1)];
      const int32_t* cap = mat == 0 ? pl.vx : pl.vy;
      const float m01 = m0[ar.kdim_pad], m0b = m0[ar.kdim_pad + 1];
      const int kb = r0 / 2 + 1;   // frequency of tile rows 0 (cos) and 1 (sin)
      float* part = reinterpret_cast<float*>(ws + ar.off_part) + ((size_t)mat * ar.rtiles + rt) * pl.V;
      for (int pc = cs; pc < ce; pc += kCornerCache) {
        const int pn = min(kCornerCache, ce - pc);
        asm volatile("bar.sync 1, %0;" ::"n"(kGen) : "memory");   // zs written / previous piece read
        for (int i = tid; i < pn; i += kGen) {
          const int vv = gr.perm[pc + i];
          sc[i] = make_int4(vv, __ldg(cap + vv), __ldg(cbp + vv) - b0, 0);
        }
        asm volatile("bar.sync 1, %0;" ::"n"(kGen) : "memory");
        // two corners per thread at a time; a frequency's (cos, sin) pair is
        // one packed FMA into a (cos, sin) sum and two packed operations of
        // angle addition
        for (int i = tid; i < pn; i += 2 * kGen) {
          const bool two = i + kGen < pn;
          const int4 e0 = sc[i], e1 = two ? sc[i + kGen] : e0;
          const uint32_t a0 = (uint32_t)e0.y, a1 = (uint32_t)e1.y;
          const int bl0 = e0.z, bl1 = e1.z;
          float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
          const float2 w0 = tl_lookup(tl, a0 & mask), w1 = tl_lookup(tl, a1 & mask);
          for (int f = 0; f < kRH; f += 8) {   // runs of 8 frequencies = 16 tile rows
            float2 v0 = tl_lookup(tl, (uint32_t)(kb + f) * a0 & mask);
            float2 v1 = tl_lookup(tl, (uint32_t)(kb + f) * a1 & mask);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
              s0 = ffma2(v0, zs[(f + t) * kVP + bl0], s0);
              s1 = ffma2(v1, zs[(f + t) * kVP + bl1], s1);
              v0 = rot2(v0, w0);
              v1 = rot2(v1, w1);
            }
          }
          const float k00 = krow ? comb[bl0] + comb[kVP + bl0] + fmaf(m0b, (float)(b0 + bl0), m01) : 0.f;
          part[e0.x] = k00 + (s0.x + s0.y);
          if (two) {
            const float k01 = krow ? comb[bl1] + comb[kVP + bl1] + fmaf(m0b, (float)(b0 + bl1), m01) : 0.f;
            part[e1.x] = k01 + (s1.x + s1.y);
          }
        }
      }
    } else {
    const uint32_t a = a_me;
    const float2 wa = tl_lookup(tl, a & mask);
    const float fb = (float)b;
    const uint32_t lane_base = ((uint32_t)(warp & 3) * 32u) << 16;
    float outv = acc0, outs = 0.f;   // cos-row and sin-row chains
    if (acc_ok) {
      for (int cb = 0; cb < kRH; cb += 32) {   // 32 rows = 16 frequencies
        const int n0 = g * kRH + cb;           // tile row of the first column
        uint32_t d1[32], d2[32];
        tmem_ld32(tmem + lane_base + (uint32_t)n0, d1);
        tmem_ld32(tmem + lane_base + (uint32_t)(kAdjPairRows + n0), d2);
        tmem_wait_ld();
        const int kb = (r0 + n0) / 2 + 1;      // rows n0 + 2 i (cos), + 1 (sin) of frequency kb + i
        float c = 0.f, sn = 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          if (i % 8 == 0) {
            const float2 an = tl_lookup(tl, (uint32_t)(kb + i) * a & mask);
            c = an.x;
            sn = an.y;
          }
          const float4 q0 = rows[n0 + 2 * i], q1 = rows[n0 + 2 * i + 1];
          const float z0 =
              fmaf(__uint_as_float(d1[2 * i]) + __uint_as_float(d2[2 * i]), q0.x, fmaf(q0.z, fb, q0.y));
          const float z1 =
              fmaf(__uint_as_float(d1[2 * i + 1]) + __uint_as_float(d2[2 * i + 1]), q1.x, fmaf(q1.z, fb, q1.y));
          outv = fmaf(c, z0, outv);
          outs = fmaf(sn, z1, outs);
          const float c1 = fmaf(c, wa.x, -(sn * wa.y)), s1 = fmaf(sn, wa.x, c * wa.y);
          c = c1;
          sn = s1;
        }
      }
    }
    outv += outs;
    if (g == 1) comb[cidx] = outv;
    asm volatile("bar.sync 1, %0;" ::"n"(kGen) : "memory");
    if (g == 0 && live) {
      float tot = outv + comb[cidx];
      if (krow) tot += fmaf(m0[ar.kdim_pad + 1], fb, m0[ar.kdim_pad]);
      reinterpret_cast<float*>(ws + ar.off_part)[((size_t)mat * ar.rtiles + rt) * pl.V + v] = tot;
    }
    }
  }

  // the pair's MMAs, commits and arrivals reach both CTAs: neither releases
  // its TMEM or leaves before both are done
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();
  if (warp == GW) {
    __syncwarp();   // lane 0 ran the MMA loop alone; dealloc is warp-collective
    tc_fence_after();
    tmem_dealloc_pair(tmem, 2 * kAdjPairRows);
  }
}

}  // namespace

cudaError_t launch_adj_tc(const AdjTcArgs& ar, const CUtensorMap& mhi, const CUtensorMap& mlo, void* ws,
                          cudaStream_t st) {
  if (ar.pl.logT > 16) return cudaErrorInvalidValue;   // the two-level table holds T <= 2^16
  auto kern = ar.grouped ? adj_tc_kernel<true> : adj_tc_kernel<false>;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(kern), kAdjSmem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  const long long mrows = ar.grouped ? (long long)ar.pl.T + 1 : ar.pl.V;   // corners or values of b
  cfg.gridDim = dim3((unsigned)(2 * ((mrows + 2 * kVP - 1) / (2 * kVP))), (unsigned)ar.rtiles, 2);
  cfg.blockDim = dim3(kThreadsA);
  cfg.dynamicSmemBytes = kAdjSmem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, mhi, mlo, ar, static_cast<uint8_t*>(ws));
  count_launch(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace fcfs
