// Continuous Haar transform of a clip (Sec. II-C), the transform the PCHT of
// Sec. III-B computes, up to level J on the tile [0, N) x [0, N), N = T:
//
//   W[0][0]                  = <f, phi_000>         = area / N
//   W[2^j + kx][ky]          = <f, psi^(hg)_{j,kx,ky}> = (2^j / N)(A00 + A01 - A10 - A11)
//   W[kx][2^j + ky]          = <f, psi^(gh)_{j,kx,ky}> = (2^j / N)(A00 - A01 + A10 - A11)
//   W[2^j + kx][2^j + ky]    = <f, psi^(hh)_{j,kx,ky}> = (2^j / N)(A00 - A01 - A10 + A11)
//
// for 0 <= j < J, 0 <= kx, ky < 2^j, with A_nm the areas of the image inside the
// four children [(2kx+n) s, (2kx+n+1) s) x [(2ky+m) s, (2ky+m+1) s) of side
// s = N / 2^(j+1) (the Haar filters g = (1, 1)/sqrt 2, h = (1, -1)/sqrt 2 acting on
// the level-(j+1) scaling coefficients (2^(j+1) / N) A_nm; first letter along x).
//
// GPU form.  The paper recurses over dyadic squares per polygon, prunes squares
// that lie completely inside or outside, and takes each square's area from the
// polygon's edges (Alg. 1).  Here every coefficient comes from the areas of the
// level-J cells (side w = N / 2^J), all of them at once:
//  * The corner form of Lemma polyip with the tail primitive makes the image the
//    signed sum of quadrants [x_v, N) x [y_v, N).  Along x a quadrant covers cell
//    i over w for i > c = floor(x_v / w), over r = (c + 1) w - x_v for i = c and
//    not at all below: the inclusive prefix sum of the two-point splat r at c,
//    w - r at c + 1.  So the cell areas are the 2-D inclusive prefix sum of
//        Z = sum_v s_v (r e_c + (w - r) e_{c+1}) (q e_d + (w - q) e_{d+1})^T
//    (points past the grid dropped).
//  * Row scans, then column scans, give the exact integer areas A_J.
//  * A pyramid of 2 x 2 sums gives the coarser areas and the three signed sums
//    per parent; each is an integer times 2^(j - log2 N), exact in FP64.
// Kernels: the corners grouped by x (count, scan, scatter); each row of Z built
// in shared memory from the corners of its own and the previous cell row,
// scanned there and written once (one CTA per row); column sums per (strip of
// 32 columns, row segment); the column scan fused with the pyramid of each
// 32 x 32 tile (five levels; one warp per strip segment); then pyramid passes
// on the coarse area grids until one cell is left.  Everything is exact
// integer arithmetic; the FP64 coefficients are assembled from their bits.
//
// Element type of Z.  No value held in Z after any of its passes is a running
// area: a row-scanned entry is the difference of two vertically adjacent cell
// areas, a fully scanned one a cell area, so |value| <= w^2, and a 32 x 32
// tile's area is at most (32 w)^2.  For w <= 1024 all of them fit in int32 and
// Z, its scans and the tile pyramid run in 32-bit integers (half the bytes and
// the instructions); intermediate sums of the row atomics and the scans may
// wrap, which two's-complement addition undoes exactly.  Larger cells use int64.
// The coarse area grids are int64 throughout.
#include <type_traits>

#include "fcfs_group.cuh"
#include "fcfs_launch.cuh"

namespace fcfs {

namespace {

constexpr int kHT = 32;          // pyramid tile side (five levels per pass)
constexpr int kHThreads = 256;
constexpr int kHaarMaxJ = 14;    // 2^28 cells: 1-2 GiB of cell areas, 2 GiB of FP64 output
constexpr int kNarrowMaxW = 1024;   // cell side up to which Z is int32
constexpr int kBand = 32;          // banded path: cell rows per band (one tile row)
constexpr int kChunk = 256;        // banded path: columns per chunk (eight 32 x 32 tiles)
constexpr int kBandStage = 4096;   // banded path: splats staged in shared memory per CTA
constexpr int kBandMaxChunks = 64; // banded path: chunks per CTA (2^14 / kChunk)

struct HaarPlan {
  int J, logN, G, N;
  int64_t V;
  int narrow;                    // 1: Z in int32 (cell side <= kNarrowMaxW)
  int strips, segs, tiles_per_seg;
  int npass;                     // pyramid passes, the fused one first; pass p leaves a grid of coarse_side[p]
  int banded;                    // 1: bands of 32 rows, the cell grid kept on chip (grids of >= 256 cells a side)
  int nbands, band_cpc, band_nq; // bands, chunks of 256 columns per CTA, CTAs per band
  int ny_pad;                    // T + 1 rounded up to 64 (the grouping's exponent array)
  size_t off_z, off_colsum, off_coarse[6], off_groups, total;
  int coarse_side[6];
};

int ilog2(long long v) {
  int r = 0;
  while ((1LL << (r + 1)) <= v) ++r;
  return r;
}

fcfs_status make_haar_plan(int64_t V, int32_t T, int32_t J, HaarPlan& hp) {
  memset(&hp, 0, sizeof(hp));
  if (T < 4 || T > 65536 || (T & (T - 1)) != 0) return FCFS_EUNSUPPORTED;
  const int logN = ilog2(T);
  if (J < 0 || J > logN || J > kHaarMaxJ) return FCFS_EUNSUPPORTED;
  if (V < 0 || V >= (1LL << 31)) return FCFS_EINVAL;
  hp.J = J;
  hp.logN = logN;
  hp.N = T;
  hp.V = V;
  hp.G = 1 << J;
  hp.narrow = (T >> J) <= kNarrowMaxW ? 1 : 0;
  const size_t elem = hp.narrow ? 4 : 8;
  const int t = hp.G < kHT ? hp.G : kHT;
  const int tiles = hp.G / t;
  hp.strips = tiles;
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // row segments: about 24 warps per SM for the fused column scan (each warp
  // walks its segment's tiles one after another)
  int segs = (24 * sms + hp.strips - 1) / hp.strips;
  segs = segs < 1 ? 1 : (segs > tiles ? tiles : segs);
  hp.tiles_per_seg = (tiles + segs - 1) / segs;
  hp.segs = (tiles + hp.tiles_per_seg - 1) / hp.tiles_per_seg;
  hp.banded = (hp.narrow && hp.G >= kChunk) ? 1 : 0;
  if (hp.banded) {
    // CTAs per band: a power of two giving at least 8 per SM over the grid
    hp.nbands = hp.G / kBand;
    const int nchunks = hp.G / kChunk;
    int nq = 1;
    while (nq < nchunks && (long long)nq * hp.nbands < 8LL * sms) nq <<= 1;
    hp.band_nq = nq;
    hp.band_cpc = nchunks / nq;
  }
  size_t o = 256;   // header: the status word
  hp.off_z = o;
  if (!hp.banded) o = align_up(o + (size_t)hp.G * hp.G * elem, kWsAlign);
  hp.off_colsum = o;
  o = align_up(o + (hp.banded ? (size_t)hp.nbands * hp.G * 4 : (size_t)hp.segs * hp.G * elem), kWsAlign);
  int side = tiles;   // side of the area grid each pass leaves, down to one cell
  for (;;) {
    hp.coarse_side[hp.npass] = side;
    hp.off_coarse[hp.npass] = o;
    o = align_up(o + (size_t)side * side * 8, kWsAlign);
    ++hp.npass;
    if (side == 1) break;
    side = side / (side < kHT ? side : kHT);
  }
  hp.ny_pad = (T + 1 + 63) / 64 * 64;
  hp.off_groups = o;
  o = align_up(o + group_bytes(V, T, hp.ny_pad), kWsAlign);
  hp.total = o;
  return FCFS_OK;
}

template <typename E>
__device__ __forceinline__ E warp_incl_scan(E v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const E t = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += t;
  }
  return v;
}

template <typename E>
__device__ __forceinline__ E warp_sum(E v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

// 32-bit sums wrap (modulo 2^32) instead of overflowing
__device__ __forceinline__ int wadd(int a, int b) { return (int)((unsigned)a + (unsigned)b); }
__device__ __forceinline__ long long wadd(long long a, long long b) { return a + b; }

// Rows [i0, i0 + nb) of Z (i0 = nb blockIdx.x) summed, built and scanned along
// the row in shared memory, written once as row blockIdx.x.  Along x the
// quadrant of a corner in cell row c = floor(x / w) covers row c over
// r = (c + 1) w - x and every later row over w: after the column scan that is
// the two-point splat r at c, w - r at c + 1.  So row i receives the corners of
// rows i (weight r) and i - 1 (weight w - r), found through the grouping of the
// corners by x, each splatted along y as q at d = floor(y / w) and w - q at
// d + 1; the inclusive scan along the row follows.  Corners with x or y
// outside [0, N) or a sign other than +-1 add nothing.  One CTA per row (nb = 1:
// the rows of Z) or per band of rows (their column sums); the scan is done by
// warps over chunks of 32 (conflict-free reads).
template <typename E>
__global__ void __launch_bounds__(kHThreads) haar_row_build_kernel(const int32_t* __restrict__ x,
                                                                   const int32_t* __restrict__ y,
                                                                   const int8_t* __restrict__ s,
                                                                   const int* __restrict__ start,
                                                                   const int* __restrict__ perm, int N, int G,
                                                                   int lw, int nb, E* Z) {
  griddep_wait();   // launched behind the grouping (programmatic dependent launch)
  using U = typename std::conditional<sizeof(E) == 4, unsigned, unsigned long long>::type;
  constexpr int kWarps = kHThreads / 32;
  extern __shared__ __align__(16) unsigned char hraw[];
  U* row = reinterpret_cast<U*>(hraw);
  __shared__ U tot[kWarps];
  const int i0 = blockIdx.x * nb;
  const long long w = 1LL << lw;
  for (int j = threadIdx.x; j < G; j += blockDim.x) row[j] = 0;
  __syncthreads();
  const int xlo = (i0 > 0 ? i0 - 1 : 0) << lw;
  const int xhi = min(N, (i0 + nb) << lw);   // corners with x in [xlo, xhi): rows i0 - 1 .. i0 + nb - 1
  const int b0 = start[xlo], e0 = start[xhi];
  for (int j = b0 + (int)threadIdx.x; j < e0; j += blockDim.x) {
    const int v = perm[j];
    const int xv = __ldg(x + v), yv = __ldg(y + v), sv = __ldg(s + v);
    if (yv < 0 || yv >= N || (sv != 1 && sv != -1)) continue;
    const int c = xv >> lw;
    const long long r = (long long)(c + 1) * w - xv;   // in (0, w]
    const long long wx = (c >= i0 ? r : 0) + (c + 1 < i0 + nb ? w - r : 0);
    if (wx == 0) continue;
    const int d = yv >> lw;
    const long long q = (long long)(d + 1) * w - yv;
    atomicAdd(&row[d], (U)(sv * wx * q));
    if (q < w && d + 1 < G) atomicAdd(&row[d + 1], (U)(sv * wx * (w - q)));
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seg = (G + kWarps - 1) / kWarps;
  const int b = warp * seg, e = min(G, b + seg);
  U sum = 0;
  for (int j = b + lane; j < e; j += 32) sum += row[j];
  sum = warp_sum(sum);
  if (lane == 0) tot[warp] = sum;
  __syncthreads();
  U off = 0;
  for (int w2 = 0; w2 < warp; ++w2) off += tot[w2];
  U* out = reinterpret_cast<U*>(Z) + (size_t)blockIdx.x * G;
  for (int j0 = b; j0 < e; j0 += 32) {   // warp-uniform
    const int j = j0 + lane;
    U v = j < e ? row[j] : 0;
    v = warp_incl_scan(v, lane);
    if (j < e) out[j] = v + off;
    off += __shfl_sync(0xffffffffu, v, 31);
  }
}

// colsum[seg][col] = sum of Z over the rows of segment seg, for the 32 columns
// of strip blockIdx.x (modulo the width of E: only differences of them are used).
template <typename E>
__global__ void __launch_bounds__(kHThreads) haar_colsum_kernel(const E* __restrict__ Z, int G, int rows_per_seg,
                                                                E* colsum) {
  griddep_wait();   // launched behind the row build
  using U = typename std::conditional<sizeof(E) == 4, unsigned, unsigned long long>::type;
  __shared__ U part[kHThreads / 32][kHT];
  const int t = G < kHT ? G : kHT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int col = blockIdx.x * t + lane;
  const int r0 = blockIdx.y * rows_per_seg, r1 = min(G, r0 + rows_per_seg);
  const U* Zu = reinterpret_cast<const U*>(Z);
  U sum = 0;
  if (lane < t)
    for (int r = r0 + warp; r < r1; r += kHThreads / 32) sum += Zu[(size_t)r * G + col];
  part[warp][lane] = sum;
  __syncthreads();
  if (warp == 0 && lane < t) {
    U tsum = 0;
    for (int w2 = 0; w2 < kHThreads / 32; ++w2) tsum += part[w2][lane];
    reinterpret_cast<U*>(colsum)[(size_t)blockIdx.y * G + col] = tsum;
  }
}

// num * 2^e as an IEEE-754 binary64 value, built from the format's fields with
// integer operations only (GB300 runs FP64 conversions and scaling at a small
// fraction of its integer rate): the sign bit, the biased exponent of the
// leading one, and the bits below the leading one as the 52-bit fraction.
// Exact for |num| < 2^53; the numerators here are at most 4 N^2 <= 2^34 and
// the exponents stay in the normal range (e >= -16).
__device__ __forceinline__ double dyadic(long long num, int e) {
  if (num == 0) return 0.0;
  const unsigned long long sign = num < 0 ? (1ULL << 63) : 0ULL;
  const unsigned long long m = num < 0 ? (unsigned long long)(-num) : (unsigned long long)num;
  const int msb = 63 - __clzll((long long)m);
  const unsigned long long frac = ((m << (63 - msb)) << 1) >> 12;
  const unsigned long long expo = (unsigned long long)(msb + e + 1023) << 52;
  return __longlong_as_double((long long)(sign | expo | frac));
}
// the same for |num| < 2^31: the fraction is the bits below the leading one
// shifted up to 52 bits, split into the two 32-bit halves of the value
__device__ __forceinline__ double dyadic(int num, int e) {
  if (num == 0) return 0.0;
  const unsigned sign = num < 0 ? 0x80000000u : 0u;
  const unsigned m = num < 0 ? (unsigned)(-num) : (unsigned)num;
  const int msb = 31 - __clz(m);
  const unsigned long long frac = (unsigned long long)(m ^ (1u << msb)) << (52 - msb);
  const unsigned hi = sign | ((unsigned)(msb + e + 1023) << 20) | (unsigned)(frac >> 32);
  return __hiloint2double((int)hi, (int)(unsigned)frac);
}

// One parent (p, q) at level j: its three wavelet coefficients go to W and its
// area is returned.  a holds the children (level j + 1 areas); (ti, tj) is the
// tile, h its parents per side at this level; W has side WG <= 2^14, so its
// offsets fit in 32 bits.
template <typename E>
__device__ __forceinline__ E parent(E (*a)[kHT + 1], int p, int q, int ti, int tj, int h, int j, int logN, double* W,
                                    int WG) {
  const E a00 = a[2 * p][2 * q], a01 = a[2 * p][2 * q + 1];
  const E a10 = a[2 * p + 1][2 * q], a11 = a[2 * p + 1][2 * q + 1];
  const unsigned P = 1u << j;
  const unsigned kx = (unsigned)(ti * h + p), ky = (unsigned)(tj * h + q);
  const int e = j - logN;
  W[(P + kx) * (unsigned)WG + ky] = dyadic((E)((a00 + a01) - (a10 + a11)), e);
  W[kx * (unsigned)WG + P + ky] = dyadic((E)((a00 - a01) + (a10 - a11)), e);
  W[(P + kx) * (unsigned)WG + P + ky] = dyadic((E)((a00 - a01) - (a10 - a11)), e);
  return (a00 + a01) + (a10 + a11);
}

// Reduce the t x t tile of level-L cell areas in a[][] through log2 t levels:
// the wavelet coefficients of levels L - 1 .. L - log2 t go to W (side WG), and
// a[0][0] ends as the tile's area.  (ti, tj): the tile's position in tiles.
// Levels with more than 64 parents use the whole CTA; warp 0 finishes the
// rest alone (threads of the other warps return at once).
__device__ void tile_pyramid(long long (*a)[kHT + 1], int t, int ti, int tj, int L, int logN, double* W, int WG) {
  const int tid = threadIdx.x;
  int cl = L, sd = t;
  for (; sd > 1 && (sd >> 1) * (sd >> 1) > 64; sd >>= 1, --cl) {
    const int h = sd >> 1;
    const bool act = tid < h * h;
    const int p = act ? tid / h : 0, q = act ? tid % h : 0;
    const long long area = act ? parent(a, p, q, ti, tj, h, cl - 1, logN, W, WG) : 0;
    __syncthreads();
    if (act) a[p][q] = area;
    __syncthreads();
  }
  if (tid >= 32) return;
  for (; sd > 1; sd >>= 1, --cl) {
    const int h = sd >> 1, np = h * h;   // at most 64 parents: two per lane
    long long ar[2] = {0, 0};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int idx = tid + 32 * u;
      if (idx < np) ar[u] = parent(a, idx / h, idx % h, ti, tj, h, cl - 1, logN, W, WG);
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int idx = tid + 32 * u;
      if (idx < np) a[idx / h][idx % h] = ar[u];
    }
    __syncwarp();
  }
}

// The t x t tile in a[][] (the warp's own shared memory) reduced through
// log2 t levels by one warp (up to 256 parents a level: eight per lane);
// a[0][0] ends as the tile's area.
template <typename E>
__device__ void warp_pyramid(E (*a)[kHT + 1], int t, int ti, int tj, int L, int logN, double* W, int WG, int lane) {
  int cl = L;
  for (int sd = t; sd > 1; sd >>= 1, --cl) {
    const int h = sd >> 1, lh = __ffs(h) - 1, np = h * h;
    E ar[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = lane + 32 * u;
      ar[u] = idx < np ? parent(a, idx >> lh, idx & (h - 1), ti, tj, h, cl - 1, logN, W, WG) : (E)0;
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = lane + 32 * u;
      if (idx < np) a[idx >> lh][idx & (h - 1)] = ar[u];
    }
    __syncwarp();
  }
}

constexpr int kStripWarps = 8;

template <typename E>
size_t strip_smem_bytes() { return (size_t)kStripWarps * kHT * (kHT + 1) * sizeof(E); }

// Column scan of the row-scanned Z fused with the pyramid of its tiles.  One
// warp per (strip of t columns, segment of tiles_per_seg tile rows), no block
// barrier: lane c owns column c of the strip.  Per tile it loads its t values
// (independent loads), adds them down the column in registers from the carry
// (the column sums of the segments above, then of the tiles done), stages the
// tile in the warp's shared memory and reduces it (levels J - 1 .. J - log2 t).
// The tile's area goes to coarse; with a single tile, W[0][0] too.
template <typename E>
__global__ void __launch_bounds__(kStripWarps * 32, sizeof(E) == 4 ? 3 : 2) haar_strip_kernel(const E* __restrict__ Z, int G, int J, int logN,
                                                                     const E* __restrict__ colsum, int strips,
                                                                     int segs, int tiles_per_seg, long long* coarse,
                                                                     double* W) {
  griddep_wait();   // launched behind the column sums
  extern __shared__ __align__(16) unsigned char hsm_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kStripWarps + warp;
  if (gw >= strips * segs) return;   // whole warps; nothing below waits on other warps
  E(*a)[kHT + 1] = reinterpret_cast<E(*)[kHT + 1]>(hsm_raw + (size_t)warp * kHT * (kHT + 1) * sizeof(E));
  const int t = G < kHT ? G : kHT;
  const int tiles = G / t;
  const int tj = gw % strips, sg = gw / strips;
  const int ti0 = sg * tiles_per_seg, ti1 = min(tiles, ti0 + tiles_per_seg);
  const bool col_ok = lane < t;
  E carry = 0;
  if (col_ok)
    for (int s2 = 0; s2 < sg; ++s2) carry = wadd(carry, colsum[(size_t)s2 * G + tj * t + lane]);
  // the tile's column values: loaded one tile ahead, so that the loads of tile
  // ti + 1 are in flight while tile ti is reduced
  E v[kHT];
  auto fetch = [&](int ti) {
    const E* src = Z + (size_t)ti * t * G + (size_t)tj * t + lane;
#pragma unroll
    for (int r = 0; r < kHT; ++r) v[r] = (col_ok && r < t) ? src[(size_t)r * G] : (E)0;
  };
  if (ti0 < ti1) fetch(ti0);
  for (int ti = ti0; ti < ti1; ++ti) {
    __syncwarp();   // lane 0's read of the previous tile's a[0][0] is done
#pragma unroll
    for (int r = 0; r < kHT; ++r) {
      carry = wadd(carry, v[r]);
      if (col_ok && r < t) a[r][lane] = carry;
    }
    __syncwarp();
    if (ti + 1 < ti1) fetch(ti + 1);
    warp_pyramid(a, t, ti, tj, J, logN, W, G, lane);
    if (lane == 0) {
      const long long area = (long long)a[0][0];
      coarse[(size_t)ti * tiles + tj] = area;
      if (tiles == 1) W[0] = dyadic(area, -logN);
    }
  }
}

// Banded path (grids of at least 256 x 256 cells, Z in 32 bits).  The cell
// areas of band b (cell rows [32 b, 32 b + 32)) at column d are
//     A(i, d) = C_b(d) + sum_{i' = 32 b}^{i} R(i', d),   R(i', d) = sum_{d' <= d} Z(i', d'),
// with C_b(d) the sum of R over all rows above the band.  The band sums S_b(d)
// (the row build with nb = 32: the rows of a band summed, then scanned) and
// their exclusive scan over the bands give C_b; each band is then built chunk
// by chunk in shared memory (row scans carried across the chunks), scanned down
// its columns from C_b and reduced by the tile pyramids, so the 2^2J cell
// areas never reach global memory.

// C_b(d) = sum over the bands b' < b of S_b'(d), in place (modulo 2^32: only
// differences matter).  One CTA per strip of 32 columns, each warp a range of
// bands: the ranges' sums, their prefix across the warps, then the running sums.
__global__ void __launch_bounds__(kHThreads) haar_band_scan_kernel(unsigned* S, int G, int nbands) {
  griddep_wait();   // launched behind the band sums
  constexpr int kWarps = kHThreads / 32;
  __shared__ unsigned tot[kWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t col = (size_t)blockIdx.x * 32 + lane;
  const int per = (nbands + kWarps - 1) / kWarps;
  const int b0 = min(nbands, warp * per), b1 = min(nbands, b0 + per);
  unsigned sum = 0;
#pragma unroll 8
  for (int b = b0; b < b1; ++b) sum += S[(size_t)b * G + col];
  tot[warp][lane] = sum;
  __syncthreads();
  unsigned run = 0;
  for (int w2 = 0; w2 < warp; ++w2) run += tot[w2][lane];
#pragma unroll 8
  for (int b = b0; b < b1; ++b) {
    const size_t o = (size_t)b * G + col;
    const unsigned v = S[o];
    S[o] = run;
    run += v;
  }
}

// f(row - i0, column, weight) for every splat of the corners of cell rows
// [i0 - 1, i0 + kBand) on the rows of the band [i0, i0 + kBand): the same terms
// as the row build's (row c with r, row c + 1 with w - r; column d with q,
// column d + 1 with w - q; empty or out-of-grid terms left out).
template <typename F>
__device__ __forceinline__ void band_splats(const int32_t* __restrict__ x, const int32_t* __restrict__ y,
                                            const int8_t* __restrict__ s, const int* __restrict__ start,
                                            const int* __restrict__ perm, int N, int G, int lw, int i0, F&& f) {
  const int w = 1 << lw;
  const int xlo = (i0 > 0 ? i0 - 1 : 0) << lw;
  const int xhi = min(N, (i0 + kBand) << lw);
  const int b0 = start[xlo], e0 = start[xhi];
  for (int j = b0 + (int)threadIdx.x; j < e0; j += blockDim.x) {
    const int v = perm[j];
    const int xv = __ldg(x + v), yv = __ldg(y + v), sv = __ldg(s + v);
    if (yv < 0 || yv >= N || (sv != 1 && sv != -1)) continue;
    const int c = xv >> lw, d = yv >> lw;
    const int r = ((c + 1) << lw) - xv, q = ((d + 1) << lw) - yv;   // in (0, w]
    const bool two = q < w && d + 1 < G;
    if (c >= i0) {
      f(c - i0, d, sv * r * q);
      if (two) f(c - i0, d + 1, sv * r * (w - q));
    }
    if (c + 1 < i0 + kBand && r < w) {
      f(c + 1 - i0, d, sv * (w - r) * q);
      if (two) f(c + 1 - i0, d + 1, sv * (w - r) * (w - q));
    }
  }
}

// the chunk's eight 32 x 33 tiles, each 4 words further along the banks than
// the last: the row scans' lanes (8 tiles x 4 rows at one column) hit distinct banks
constexpr int kBandTileWords = kHT * (kHT + 1) + 4;
constexpr size_t kBandTiles = (size_t)(kChunk / kHT) * kBandTileWords * 4;
constexpr size_t kBandSmem = kBandTiles + (size_t)kBandStage * 8;

// One CTA per (band, range of cpc chunks of 256 columns), 8 warps.  The band's
// splats left of the range are summed into the row carries, those in it staged
// in shared memory by chunk (counting sort; a band with more than kBandStage of
// them splats each chunk straight from the corners instead).  Per chunk: the
// splats into eight 32 x 32 tiles, the row scans from the row carries (thread
// (row, tile): its 32 columns in order, the tiles' totals prefixed across the
// row's eight threads), then per warp its tile's column scan from C_b and the
// tile pyramid (levels J - 1 .. J - 5), the tile's area to the coarse grid.
__global__ void __launch_bounds__(kHThreads, 3) haar_band_kernel(
    const int32_t* __restrict__ x, const int32_t* __restrict__ y, const int8_t* __restrict__ s,
    const int* __restrict__ start, const int* __restrict__ perm, int N, int G, int lw, int J, int logN,
    const unsigned* __restrict__ C, int cpc, long long* coarse, double* W) {
  griddep_wait();   // launched behind the band scan (and the grouping before it)
  extern __shared__ __align__(16) unsigned char bsm[];
  auto tile = [&](int t) { return reinterpret_cast<unsigned(*)[kHT + 1]>(bsm + (size_t)t * kBandTileWords * 4); };
  uint2* stage = reinterpret_cast<uint2*>(bsm + kBandTiles);   // {row << 8 | column in chunk, weight}
  __shared__ unsigned rowcarry[kBand];
  __shared__ int off[kBandMaxChunks + 1], cur[kBandMaxChunks];
  const int b = blockIdx.y, i0 = b * kBand;
  const int d0 = blockIdx.x * cpc * kChunk, d1 = d0 + cpc * kChunk;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid < kBand) rowcarry[tid] = 0;
  if (tid <= kBandMaxChunks) off[tid] = 0;
  __syncthreads();
  band_splats(x, y, s, start, perm, N, G, lw, i0, [&](int rl, int col, int wt) {
    if (col < d0) atomicAdd(&rowcarry[rl], (unsigned)wt);
    else if (col < d1) atomicAdd(&off[(col - d0) / kChunk], 1);
  });
  __syncthreads();
  if (tid == 0) {
    int o = 0;
    for (int k = 0; k < cpc; ++k) {
      const int c = off[k];
      off[k] = cur[k] = o;
      o += c;
    }
    off[cpc] = o;
  }
  __syncthreads();
  const bool staged = off[cpc] <= kBandStage;   // block-uniform
  if (staged) {
    band_splats(x, y, s, start, perm, N, G, lw, i0, [&](int rl, int col, int wt) {
      if (col >= d0 && col < d1) {
        const int pos = atomicAdd(&cur[(col - d0) / kChunk], 1);
        stage[pos] = make_uint2((unsigned)(rl << 8) | (unsigned)((col - d0) % kChunk), (unsigned)wt);
      }
    });
  }
  for (int k = 0; k < cpc; ++k) {
    const int c0 = d0 + k * kChunk;
    __syncthreads();   // the previous chunk's pyramids (and the staging) are done
    uint4* tz = reinterpret_cast<uint4*>(bsm);
    for (int e = tid; e < (int)(kBandTiles / 16); e += kHThreads) tz[e] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    if (staged) {
      for (int e = off[k] + tid; e < off[k + 1]; e += kHThreads) {
        const uint2 st = stage[e];
        const int rl = (int)(st.x >> 8), cl = (int)(st.x & 255u);
        atomicAdd(&tile(cl >> 5)[rl][cl & 31], st.y);
      }
    } else {
      band_splats(x, y, s, start, perm, N, G, lw, i0, [&](int rl, int col, int wt) {
        if (col >= c0 && col < c0 + kChunk) atomicAdd(&tile((col - c0) >> 5)[rl][(col - c0) & 31], (unsigned)wt);
      });
    }
    __syncthreads();
    {
      // row scans: thread (row rl, tile t) sums its 32 columns, the totals of the
      // row's tiles are prefixed over its eight consecutive lanes, then the
      // running sums are written from the row carry plus that prefix
      const int rl = tid >> 3, t = tid & 7;
      unsigned(*row)[kHT + 1] = tile(t);
      unsigned sum = 0;
#pragma unroll 8
      for (int c = 0; c < kHT; ++c) sum += row[rl][c];
      unsigned incl = sum;
#pragma unroll
      for (int d = 1; d < 8; d <<= 1) {
        const unsigned u = __shfl_up_sync(0xffffffffu, incl, d, 8);
        if (t >= d) incl += u;
      }
      unsigned run = rowcarry[rl] + (incl - sum);
#pragma unroll 8
      for (int c = 0; c < kHT; ++c) {
        run += row[rl][c];
        row[rl][c] = run;
      }
      __syncthreads();   // every thread has read its row carry
      if (t == 7) rowcarry[rl] = run;
    }
    __syncthreads();
    // the warp's tile: column scan from C_b, then its pyramid
    int(*a)[kHT + 1] = reinterpret_cast<int(*)[kHT + 1]>(tile(warp));
    unsigned carry = C[(size_t)b * G + c0 + warp * kHT + lane];
#pragma unroll
    for (int r = 0; r < kHT; ++r) {
      carry += (unsigned)a[r][lane];
      a[r][lane] = (int)carry;
    }
    __syncwarp();
    const int tj = c0 / kHT + warp;
    warp_pyramid(a, kHT, b, tj, J, logN, W, G, lane);
    if (lane == 0) coarse[(size_t)b * (G / kHT) + tj] = (long long)a[0][0];
  }
}

// One CTA per t x t tile of a coarse area grid of side G (cells of level L):
// the tile's levels L - 1 .. L - log2 t; its area goes to coarse[ti][tj], and
// the last pass (a single tile) writes W[0][0] = area / N.
__global__ void __launch_bounds__(kHThreads) haar_coarse_kernel(const long long* __restrict__ A, int G, int L,
                                                                int logN, long long* coarse, double* W, int WG) {
  griddep_wait();   // launched behind the previous pyramid pass
  __shared__ long long a[kHT][kHT + 1];
  const int t = G < kHT ? G : kHT;
  const int tiles = G / t;
  const int tid = threadIdx.x;
  const int ti = blockIdx.x / tiles, tj = blockIdx.x % tiles;
#pragma unroll
  for (int k = 0; k < kHT * kHT / kHThreads; ++k) {
    const int r = (tid >> 5) + (kHThreads / 32) * k, c = tid & 31;
    if (r < t && c < t) a[r][c] = A[(size_t)(ti * t + r) * G + tj * t + c];
  }
  __syncthreads();
  tile_pyramid(a, t, ti, tj, L, logN, W, WG);
  if (tid == 0) {
    const long long area = a[0][0];
    coarse[(size_t)ti * tiles + tj] = area;
    if (tiles == 1) W[0] = dyadic(area, -logN);
  }
}

template <typename E>
cudaError_t launch_haar_t(const HaarPlan& hp, const int32_t* x, const int32_t* y, const int8_t* s, uint8_t* ws,
                          double* W, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(ws, 0, 256, st);   // the header (status word)
  if (e != cudaSuccess) return e;
  E* Z = reinterpret_cast<E*>(ws + hp.off_z);
  const int G = hp.G, t = G < kHT ? G : kHT;
  // the corners grouped by x (counting sort), then every row of Z built once
  uint8_t* gb = ws + hp.off_groups;
  if ((e = launch_grouping(x, nullptr, hp.V, hp.N, hp.ny_pad, gb, st)) != cudaSuccess) return e;
  const Groups g = groups_at(gb, hp.N, hp.ny_pad);
  const size_t row_smem = (size_t)G * sizeof(E);
  const int lw = hp.logN - hp.J;
  long long* coarse = reinterpret_cast<long long*>(ws + hp.off_coarse[0]);
  ensure_smem(reinterpret_cast<const void*>(haar_row_build_kernel<E>), row_smem);
  if (hp.banded) {
    // band sums, their scan over the bands, then the bands on chip
    unsigned* S = reinterpret_cast<unsigned*>(ws + hp.off_colsum);
    if ((e = launch_after(haar_row_build_kernel<E>, dim3(hp.nbands), dim3(kHThreads), row_smem, st, x, y, s,
                          (const int*)g.start, (const int*)g.perm, hp.N, G, lw, kBand,
                          reinterpret_cast<E*>(S))) != cudaSuccess)
      return e;
    if ((e = launch_after(haar_band_scan_kernel, dim3(G / 32), dim3(kHThreads), 0, st, S, G, hp.nbands)) !=
        cudaSuccess)
      return e;
    ensure_smem(reinterpret_cast<const void*>(haar_band_kernel), kBandSmem);
    if ((e = launch_after(haar_band_kernel, dim3(hp.band_nq, hp.nbands), dim3(kHThreads), kBandSmem, st, x, y, s,
                          (const int*)g.start, (const int*)g.perm, hp.N, G, lw, hp.J, hp.logN, (const unsigned*)S,
                          hp.band_cpc, coarse, W)) != cudaSuccess)
      return e;
  } else {
    if ((e = launch_after(haar_row_build_kernel<E>, dim3(G), dim3(kHThreads), row_smem, st, x, y, s,
                          (const int*)g.start, (const int*)g.perm, hp.N, G, lw, 1, Z)) != cudaSuccess)
      return e;
    E* colsum = reinterpret_cast<E*>(ws + hp.off_colsum);
    if ((e = launch_after(haar_colsum_kernel<E>, dim3(hp.strips, hp.segs), dim3(kHThreads), 0, st, Z, G,
                          hp.tiles_per_seg * t, colsum)) != cudaSuccess)
      return e;
    const int warps = hp.strips * hp.segs;
    ensure_smem(reinterpret_cast<const void*>(haar_strip_kernel<E>), strip_smem_bytes<E>());
    if ((e = launch_after(haar_strip_kernel<E>, dim3((warps + kStripWarps - 1) / kStripWarps),
                          dim3(kStripWarps * 32), strip_smem_bytes<E>(), st, (const E*)Z, G, hp.J, hp.logN,
                          (const E*)colsum, hp.strips, hp.segs, hp.tiles_per_seg, coarse, W)) != cudaSuccess)
      return e;
  }
  int L = hp.J - ilog2(t);
  for (int p = 1; p < hp.npass; ++p) {
    const int g = hp.coarse_side[p - 1], tt = g < kHT ? g : kHT;
    long long* next = reinterpret_cast<long long*>(ws + hp.off_coarse[p]);
    if ((e = launch_after(haar_coarse_kernel, dim3((g / tt) * (g / tt)), dim3(kHThreads), 0, st,
                          (const long long*)coarse, g, L, hp.logN, next, W, G)) != cudaSuccess)
      return e;
    coarse = next;
    L -= ilog2(tt);
  }
  return cudaGetLastError();
}

cudaError_t launch_haar(const HaarPlan& hp, const int32_t* x, const int32_t* y, const int8_t* s, uint8_t* ws,
                        double* W, cudaStream_t st) {
  return hp.narrow ? launch_haar_t<int>(hp, x, y, s, ws, W, st) : launch_haar_t<long long>(hp, x, y, s, ws, W, st);
}

}  // namespace

}  // namespace fcfs

using namespace fcfs;

extern "C" {

size_t fcfs_haar_workspace_size(int64_t V, int32_t T, int32_t J) {
  HaarPlan hp;
  if (make_haar_plan(V, T, J, hp) != FCFS_OK) return 0;
  return hp.total;
}

fcfs_status fcfs_haar(const int32_t* x, const int32_t* y, const int8_t* s, int64_t V, int32_t T, int32_t J,
                      uint32_t flags, double* W_out, void* workspace, size_t ws_bytes, void* stream) {
  auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (!W_out || flags != 0) return FCFS_EINVAL;
  if (V > 0 && (!x || !y || !s || !a16(x) || !a16(y) || !a16(s))) return FCFS_EINVAL;
  HaarPlan hp;
  fcfs_status r = make_haar_plan(V, T, J, hp);
  if (r != FCFS_OK) return r;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kWsAlign) != 0 || ws_bytes < hp.total)
    return FCFS_EWORKSPACE;
  if (launch_haar(hp, x, y, s, static_cast<uint8_t*>(workspace), W_out, static_cast<cudaStream_t>(stream)) !=
      cudaSuccess)
    return FCFS_ECUDA;
  return FCFS_OK;
}

}  // extern "C"
