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
//        Z = sum_v s_v (r e_c + (w - r) e_{c+1}) (q e_d + (w - q) e_{d+1})^T,
//    four integer atomics per corner (points past the grid dropped).
//  * Row scans, then column scans, give the exact int64 areas A_J.
//  * A pyramid of 2 x 2 sums gives the coarser areas and the three signed sums
//    per parent; each is an integer times 2^(j - log2 N), exact in FP64.
// Kernels: Z zeroed (memset), splat, row scan (one CTA per row), column sums
// per (strip of 32 columns, row segment), column scan fused with the pyramid
// of each 32 x 32 tile (five levels), then pyramid passes on the coarse area
// grids until one cell is left.  Everything is exact integer arithmetic.
#include "fcfs_common.cuh"

namespace fcfs {

namespace {

constexpr int kHT = 32;          // pyramid tile side (five levels per pass)
constexpr int kHThreads = 256;
constexpr int kHaarMaxJ = 14;    // 2^28 cells: 2 GiB of int64 areas, 2 GiB of FP64 output

struct HaarPlan {
  int J, logN, G, N;
  int64_t V;
  int strips, segs, tiles_per_seg;
  int npass;                     // pyramid passes, the fused one first; pass p leaves a grid of coarse_side[p]
  size_t off_z, off_colsum, off_coarse[6], total;
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
  const int t = hp.G < kHT ? hp.G : kHT;
  const int tiles = hp.G / t;
  hp.strips = tiles;
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int segs = (2 * sms + hp.strips - 1) / hp.strips;
  segs = segs < 1 ? 1 : (segs > tiles ? tiles : segs);
  hp.tiles_per_seg = (tiles + segs - 1) / segs;
  hp.segs = (tiles + hp.tiles_per_seg - 1) / hp.tiles_per_seg;
  size_t o = 256;   // header: the status word
  hp.off_z = o;
  o = align_up(o + (size_t)hp.G * hp.G * 8, kWsAlign);
  hp.off_colsum = o;
  o = align_up(o + (size_t)hp.segs * hp.G * 8, kWsAlign);
  int side = tiles;   // side of the area grid each pass leaves, down to one cell
  for (;;) {
    hp.coarse_side[hp.npass] = side;
    hp.off_coarse[hp.npass] = o;
    o = align_up(o + (size_t)side * side * 8, kWsAlign);
    ++hp.npass;
    if (side == 1) break;
    side = side / (side < kHT ? side : kHT);
  }
  hp.total = o;
  return FCFS_OK;
}

__device__ __forceinline__ void red_add(long long* p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

// Four splat weights per corner; corners outside [0, N] are dropped.
__global__ void haar_splat_kernel(const int32_t* __restrict__ x, const int32_t* __restrict__ y,
                                  const int8_t* __restrict__ s, long long V, int N, int J, int lw, long long* Z) {
  const int G = 1 << J;
  const long long w = 1LL << lw;   // cell side N / 2^J
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    const int xv = x[v], yv = y[v], sv = s[v];
    if (xv < 0 || xv >= N || yv < 0 || yv >= N || (sv != 1 && sv != -1)) continue;   // x = N: empty quadrant
    const int c = xv >> lw, d = yv >> lw;
    const long long r = (long long)(c + 1) * w - xv, q = (long long)(d + 1) * w - yv;   // in (0, w]
    long long* row = Z + (size_t)c * G;
    red_add(row + d, sv * r * q);
    if (q < w && d + 1 < G) red_add(row + d + 1, sv * r * (w - q));
    if (r < w && c + 1 < G) {
      red_add(row + G + d, sv * (w - r) * q);
      if (q < w && d + 1 < G) red_add(row + G + d + 1, sv * (w - r) * (w - q));
    }
  }
}

__device__ __forceinline__ long long warp_incl_scan(long long v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const long long t = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += t;
  }
  return v;
}

__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

// Inclusive prefix sum along every row of Z (G x G), in place.  One CTA per
// row; warp w owns the segment [w seg, (w+1) seg): it sums the segment, the
// CTA combines the eight totals, and each warp rescans its segment in chunks
// of 32 (one element per lane) from its offset.
__global__ void __launch_bounds__(kHThreads) haar_row_scan_kernel(long long* Z, int G) {
  __shared__ long long tot[kHThreads / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  long long* row = Z + (size_t)blockIdx.x * G;
  const int seg = (G + kHThreads / 32 - 1) / (kHThreads / 32);
  const int b = warp * seg, e = min(G, b + seg);
  long long sum = 0;
  for (int i = b + lane; i < e; i += 32) sum += row[i];
  sum = warp_sum(sum);
  if (lane == 0) tot[warp] = sum;
  __syncthreads();
  long long off = 0;
  for (int w2 = 0; w2 < warp; ++w2) off += tot[w2];
  for (int i0 = b; i0 < e; i0 += 32) {   // warp-uniform
    const int i = i0 + lane;
    long long v = i < e ? row[i] : 0;
    v = warp_incl_scan(v, lane);
    if (i < e) row[i] = v + off;
    off += __shfl_sync(0xffffffffu, v, 31);
  }
}

// colsum[seg][col] = sum of Z over the rows of segment seg, for the 32 columns
// of strip blockIdx.x.
__global__ void __launch_bounds__(kHThreads) haar_colsum_kernel(const long long* __restrict__ Z, int G,
                                                                int rows_per_seg, long long* colsum) {
  __shared__ long long part[kHThreads / 32][kHT];
  const int t = G < kHT ? G : kHT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int col = blockIdx.x * t + lane;
  const int r0 = blockIdx.y * rows_per_seg, r1 = min(G, r0 + rows_per_seg);
  long long sum = 0;
  if (lane < t)
    for (int r = r0 + warp; r < r1; r += kHThreads / 32) sum += Z[(size_t)r * G + col];
  part[warp][lane] = sum;
  __syncthreads();
  if (warp == 0 && lane < t) {
    long long tsum = 0;
    for (int w2 = 0; w2 < kHThreads / 32; ++w2) tsum += part[w2][lane];
    colsum[(size_t)blockIdx.y * G + col] = tsum;
  }
}

// Reduce the t x t tile of level-L cell areas in a[][] through log2 t levels:
// the wavelet coefficients of levels L - 1 .. L - log2 t go to W (side WG), and
// a[0][0] ends as the tile's area.  (ti, tj): the tile's position in tiles.
__device__ void tile_pyramid(long long (*a)[kHT + 1], int t, int ti, int tj, int L, int logN, double* W, int WG) {
  const int tid = threadIdx.x;
  int cl = L;
  for (int sd = t; sd > 1; sd >>= 1, --cl) {
    const int h = sd >> 1, j = cl - 1;
    const bool act = tid < h * h;
    const int p = act ? tid / h : 0, q = act ? tid % h : 0;
    long long area = 0;
    if (act) {
      const long long a00 = a[2 * p][2 * q], a01 = a[2 * p][2 * q + 1];
      const long long a10 = a[2 * p + 1][2 * q], a11 = a[2 * p + 1][2 * q + 1];
      area = (a00 + a01) + (a10 + a11);
      const long long P = 1LL << j;
      const long long kx = (long long)ti * h + p, ky = (long long)tj * h + q;
      const int e = j - logN;
      W[(size_t)(P + kx) * WG + ky] = ldexp((double)((a00 + a01) - (a10 + a11)), e);
      W[(size_t)kx * WG + P + ky] = ldexp((double)((a00 - a01) + (a10 - a11)), e);
      W[(size_t)(P + kx) * WG + P + ky] = ldexp((double)((a00 - a01) - (a10 - a11)), e);
    }
    __syncthreads();
    if (act) a[p][q] = area;
    __syncthreads();
  }
}

// SCAN: blockIdx = (strip, segment); the CTA walks the segment's tiles of the
// row-scanned Z from top to bottom, finishing the column scan with carries
// (the column sums of the segments above, then of the tiles it has done), and
// reduces each tile.  !SCAN: one CTA per tile of an area grid of side G.
// Each tile's area goes to coarse[ti][tj] (side G / t); the last pass (G == t)
// also writes W[0][0] = area / N.
template <bool SCAN>
__global__ void __launch_bounds__(kHThreads) haar_pyramid_kernel(const long long* __restrict__ A, int G, int L,
                                                                 int logN, const long long* __restrict__ colsum,
                                                                 int tiles_per_seg, long long* coarse, double* W,
                                                                 int WG) {
  __shared__ long long a[kHT][kHT + 1];
  __shared__ long long carry[kHT];
  const int t = G < kHT ? G : kHT;
  const int tiles = G / t;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int tj, ti0, ti1;
  if (SCAN) {
    tj = blockIdx.x;
    ti0 = blockIdx.y * tiles_per_seg;
    ti1 = min(tiles, ti0 + tiles_per_seg);
    if (tid < t) {
      long long c0 = 0;
      for (int sg = 0; sg < (int)blockIdx.y; ++sg) c0 += colsum[(size_t)sg * G + tj * t + tid];
      carry[tid] = c0;
    }
  } else {
    ti0 = blockIdx.x / tiles;
    tj = blockIdx.x % tiles;
    ti1 = ti0 + 1;
  }
  for (int ti = ti0; ti < ti1; ++ti) {
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kHT * kHT / kHThreads; ++k) {
      const int r = (tid >> 5) + (kHThreads / 32) * k, c = tid & 31;
      if (r < t && c < t) a[r][c] = A[(size_t)(ti * t + r) * G + tj * t + c];
    }
    __syncthreads();
    if (SCAN) {   // inclusive scan down each column of the tile, from the carry
      for (int cc = warp; cc < t; cc += kHThreads / 32) {
        long long v = lane < t ? a[lane][cc] : 0;
        v = warp_incl_scan(v, lane) + carry[cc];
        if (lane < t) a[lane][cc] = v;
        const long long last = __shfl_sync(0xffffffffu, v, t - 1);
        __syncwarp();
        if (lane == 0) carry[cc] = last;
      }
      __syncthreads();
    }
    tile_pyramid(a, t, ti, tj, L, logN, W, WG);
    if (tid == 0) {
      const long long area = a[0][0];
      coarse[(size_t)ti * tiles + tj] = area;
      if (tiles == 1) W[0] = ldexp((double)area, -logN);
    }
  }
}

cudaError_t launch_haar(const HaarPlan& hp, const int32_t* x, const int32_t* y, const int8_t* s, uint8_t* ws,
                        double* W, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(ws, 0, hp.off_colsum, st);   // header and Z
  if (e != cudaSuccess) return e;
  long long* Z = reinterpret_cast<long long*>(ws + hp.off_z);
  const int G = hp.G, t = G < kHT ? G : kHT;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (hp.V > 0) {
    const int blocks = (int)std::min<long long>((hp.V + 255) / 256, 8LL * sms);
    haar_splat_kernel<<<blocks, 256, 0, st>>>(x, y, s, hp.V, hp.N, hp.J, hp.logN - hp.J, Z);
    count_launch(1);
  }
  haar_row_scan_kernel<<<G, kHThreads, 0, st>>>(Z, G);
  count_launch(1);
  long long* colsum = reinterpret_cast<long long*>(ws + hp.off_colsum);
  haar_colsum_kernel<<<dim3(hp.strips, hp.segs), kHThreads, 0, st>>>(Z, G, hp.tiles_per_seg * t, colsum);
  count_launch(1);
  long long* coarse = reinterpret_cast<long long*>(ws + hp.off_coarse[0]);
  haar_pyramid_kernel<true><<<dim3(hp.strips, hp.segs), kHThreads, 0, st>>>(Z, G, hp.J, hp.logN, colsum,
                                                                            hp.tiles_per_seg, coarse, W, G);
  count_launch(1);
  int L = hp.J - ilog2(t);
  for (int p = 1; p < hp.npass; ++p) {
    const int g = hp.coarse_side[p - 1], tt = g < kHT ? g : kHT;
    long long* next = reinterpret_cast<long long*>(ws + hp.off_coarse[p]);
    haar_pyramid_kernel<false><<<(g / tt) * (g / tt), kHThreads, 0, st>>>(coarse, g, L, hp.logN, nullptr, 0, next,
                                                                         W, G);
    count_launch(1);
    coarse = next;
    L -= ilog2(tt);
  }
  return cudaGetLastError();
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
