/*
 * fcfs.h -- C ABI of the GB300 (sm_103a) continuous Fourier-series library for
 * Manhattan clips (fast continuous Fourier series, FCFS).
 *
 * The transform.  A clip is the period [0,T) x [0,T) holding disjoint simple
 * rectilinear lattice polygons (Sec. II-A.2, Eq. polydef_R); its image is the sum
 * of their indicators (Sec. III-A, Eq. signal_model).  The library returns the
 * unnormalised continuous Fourier-series block
 *
 *     F(k,l) = integral over the image of exp(-j 2 pi (k x + l y) / T) dx dy,
 *     |k|, |l| <= K,
 *
 * i.e. the paper's coefficients of Eq. fourier_basis times T, so F(0,0) is the
 * area.  Each polygon enters as its signed corners (x_v, y_v, s_v): by
 * Prop. rect_union and Lemma polyip with the tail primitive, the polygon is the
 * signed sum of upper-right quadrants [x_v,T) x [y_v,T), s_v = -1 at the start
 * and +1 at the end of every horizontal edge of a clockwise ring (y up),
 * equivalently the 2-D finite difference of the occupancy at the corner.  Then
 *
 *     F = X diag(s) Y^T,   X[k,v] = integral_{x_v}^T exp(-j 2 pi k t / T) dt,
 *
 * evaluated on the GPU in the reduced closed forms of Prop. CFT: F(0,0) is the
 * exact integer area (Eq. Fdc), F(k,0) and F(0,l) are weighted 1-D sums
 * (Eqs. Fk0, F0l), and F(k,l), k,l != 0, is -T^2/(4 pi^2 k l) times the 2-D DFT
 * of the sparse +-1 corner image at (k mod T, l mod T) (Eq. Fkl, Step 4).
 *
 * The same corner set also gives two other transforms of the clip: the
 * continuous cosine series (fcfs_cosine, the extension named in the
 * concluding section) and the continuous Haar transform that the PCHT of
 * Sec. III-B computes (fcfs_haar).
 *
 * Common conventions.
 *  - Every array pointer is a DEVICE pointer owned by the caller.  The library
 *    allocates nothing on the device; scratch memory is the caller's workspace.
 *  - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL is the
 *    legacy default stream).  Calls return once the work is enqueued.
 *  - Vertex arrays are structure-of-arrays: int32 x[V], int32 y[V], int8 s[V],
 *    16-byte aligned (torch allocations are), vertices of a polygon contiguous.
 *  - T is a power of two, 4 <= T <= 65536; coordinates satisfy 0 <= x,y <= T;
 *    s is +1 or -1; the signed set must be balanced (every vertical and every
 *    horizontal line carries signs summing to zero), as it is for any union of
 *    polygons.  1 <= K <= 4096.
 *  - F_out is complex64 interleaved (re, im), (2K+1) x (2K+1) row-major,
 *    F_out[(k+K)*(2K+1) + (l+K)] = F(k,l).
 *  - Host-detectable errors are returned at once and nothing is enqueued.
 *    Errors found on the device (bad vertex data with FCFS_FLAG_VALIDATE, a
 *    bounded wait that gave up) are written to a status word in the workspace,
 *    read with fcfs_get_status().  No kernel traps.
 *  - Results are deterministic: reductions run in a fixed order.
 */
#ifndef FCFS_H
#define FCFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FCFS_OK = 0,
    FCFS_EINVAL = 1,         /* bad scalar argument, NULL or misaligned pointer */
    FCFS_EINVAL_DATA = 2,    /* device validation rejected the vertex data */
    FCFS_EWORKSPACE = 3,     /* workspace NULL, misaligned (256 B) or too small */
    FCFS_ECUDA = 4,          /* a CUDA runtime or driver call failed */
    FCFS_ETIMEOUT = 5,       /* a bounded device-side wait gave up */
    FCFS_EUNSUPPORTED = 6    /* size or precision outside the implemented range */
} fcfs_status;

typedef enum {
    FCFS_PREC_FP32 = 0,      /* CUDA-core FP32 FMAs, FP32 sincos table */
    FCFS_PREC_SPLIT_F16 = 1  /* tcgen05 tensor cores, hi+lo FP16 operands, FP32 accumulate */
} fcfs_precision;

enum {
    FCFS_FLAG_VALIDATE = 1   /* check ranges, signs and balance on the device */
};

/* Library version, major*10000 + minor*100 + patch. */
int fcfs_version(void);

/* Human-readable name of a status code (static string). */
const char* fcfs_status_string(fcfs_status st);

/* Number of kernels this process has enqueued through the library so far
 * (host-side counter; lets a caller count launches inside a timed region). */
uint64_t fcfs_launch_count(void);

/*
 * Forward block of one clip (Prop. CFT, Alg. 2).
 *   x, y, s    : V signed corners (device), see conventions.
 *   V          : number of corners, 0 <= V < 2^31.  V = 0 gives F = 0.
 *   T, K       : period and cut-off.
 *   prec       : fcfs_precision.
 *   flags      : 0 or FCFS_FLAG_VALIDATE.
 *   F_out      : (2K+1)^2 complex64 (device), written completely.
 *   area_out   : one int64 (device), the exact area F(0,0).
 *   workspace  : device scratch, 256-byte aligned, >= fcfs_workspace_size(...)
 *                bytes; its first bytes hold the status word of this call.
 * Returns FCFS_OK once enqueued.
 */
size_t fcfs_workspace_size(int64_t V, int32_t T, int32_t K, int32_t prec);
fcfs_status fcfs_forward(const int32_t* x, const int32_t* y, const int8_t* s, int64_t V,
                         int32_t T, int32_t K, int32_t prec, uint32_t flags,
                         float* F_out, int64_t* area_out,
                         void* workspace, size_t ws_bytes, void* stream);

/*
 * Adjoint: derivatives of a real loss L with respect to every corner
 * coordinate, given the cotangent dF = dL/dRe F + j dL/dIm F over the block
 * (complex64, same layout as F_out).  Differentiating Lemma polyip with the
 * tail primitive, dX[k,v]/dx_v = -exp(-j 2 pi k x_v / T), so
 *   gx[v] = -s_v Re sum_{k,l} conj(dF(k,l)) exp(-j 2 pi k x_v/T) X[l](y_v),
 *   gy[v] = -s_v Re sum_{k,l} conj(dF(k,l)) X[k](x_v) exp(-j 2 pi l y_v/T),
 * with the full tail integrals (per corner their constant parts do not cancel).
 * Three forms (fcfs_adjoint_grouped): per corner, or with the corners grouped
 * by the contracted coordinate b (y for gx, x for gy) either a split-FP16
 * contraction over the values of b or, per frequency k, one input-pruned FFT
 * of length T along b (P = T / L FFTs of length L >= 2K, the pruned FFT of
 * Sec. III-C run on the adjoint) followed by one (K+1)-term dot per corner.
 *   gx, gy     : V floats each (device), written completely.
 * Workspace as for fcfs_forward, sized by fcfs_adjoint_workspace_size().
 */
size_t fcfs_adjoint_workspace_size(int64_t V, int32_t T, int32_t K, int32_t prec);
fcfs_status fcfs_adjoint(const int32_t* x, const int32_t* y, const int8_t* s, int64_t V,
                         int32_t T, int32_t K, int32_t prec, const float* dF,
                         float* gx, float* gy,
                         void* workspace, size_t ws_bytes, void* stream);

/*
 * Chain corner derivatives to edge positions: a vertical edge (axis 0) sits at
 * x and moves the x of both its corners, a horizontal edge (axis 1) sits at y:
 *   gE[e] = g_axis[ev0[e]] + g_axis[ev1[e]],  g_0 = gx, g_1 = gy.
 *   ev0, ev1   : E corner indices (device, int32, each < V).
 *   eaxis      : E axis codes (device, int8, 0 or 1).
 *   gE         : E floats (device).
 * Needs no workspace; indices are trusted (callers pass the rings' edges).
 */
fcfs_status fcfs_edge_chain(const float* gx, const float* gy, const int32_t* ev0,
                            const int32_t* ev1, const int8_t* eaxis, int64_t E,
                            float* gE, void* stream);

/*
 * Batch of clips sharing T and K (tiles of a layout are independent, Sec. III-A):
 * clip c owns corners [offsets[c], offsets[c+1]) of the concatenated arrays.
 *   offsets    : n_clips + 1 int64 (device), offsets[0] = 0,
 *                offsets[n_clips] = V_total, non-decreasing.
 *   F_out      : n_clips * (2K+1)^2 complex64 (device), clip-major.
 *   area_out   : n_clips int64 (device).
 * A device-built list of (clip, output tile, vertex range) units is covered
 * by one launch of the contraction kernel, so the call needs no host
 * synchronisation and can be captured in a CUDA graph.  flags must be 0.
 * Workspace sized by fcfs_batch_workspace_size(V_total, n_clips, ...).
 */
size_t fcfs_batch_workspace_size(int64_t V_total, int32_t n_clips, int32_t T, int32_t K,
                                 int32_t prec);
fcfs_status fcfs_batch(const int32_t* x, const int32_t* y, const int8_t* s,
                       const int64_t* offsets, int32_t n_clips, int64_t V_total,
                       int32_t T, int32_t K, int32_t prec, uint32_t flags,
                       float* F_out, int64_t* area_out,
                       void* workspace, size_t ws_bytes, void* stream);

/*
 * Plans: one workload's sizes and launch-shape choices in an opaque object.
 * Tiles of a layout are independent (Sec. III-A), so how the work is cut (the
 * contraction's form, its vertex splits, the tile shape, the batch unit size)
 * changes nothing in the result beyond FP32 rounding; a plan carries those
 * choices, fixed by a tuner or left to the library's rules.  A plan's calls
 * apply its knobs for their own duration on the calling thread; they ignore
 * the process-wide fcfs_debug_set_* hooks for every knob the plan sets.
 *   kind       : FCFS_PLAN_FORWARD (n_clips = 1), FCFS_PLAN_BATCH, FCFS_PLAN_ADJOINT
 *                (n_clips = 1).
 *   V          : corners (the batch total), as for the entry points.
 * fcfs_plan_create returns FCFS_EINVAL for bad arguments, FCFS_EUNSUPPORTED
 * for sizes the entry points reject, and sets *plan (else NULL); the caller
 * owns the plan and releases it with fcfs_plan_destroy.
 * Knobs (fcfs_plan_set; -1 where allowed, or 0, means automatic):
 *   FCFS_KNOB_FORM        forward: 0 over the corners, 1 corners grouped by y
 *                         with the split-FP16 contraction over y, 2 grouped with
 *                         the pruned FFT along y; adjoint: 0 per corner, 1
 *                         grouped with the split-FP16 contraction, 2 grouped
 *                         with the pruned FFT; batch: 0 direct units, 1 grouped.
 *   FCFS_KNOB_SPLITS      forward: vertex splits of the contraction.
 *   FCFS_KNOB_PAIR        forward and batch: 1 CTA-pair 256 x 256 tiles (2-SM
 *                         MMA) where eligible, 0 one-CTA tiles.
 *   FCFS_KNOB_UNIT_CHUNKS batch: pipeline chunks per (clip, tile, split) unit.
 * fcfs_plan_set returns FCFS_EINVAL for a knob the kind does not have or a
 * value out of range.  fcfs_plan_get returns the value a call will use (the
 * automatic ones resolved), -1 on error.  fcfs_plan_workspace_size is the
 * workspace for the plan's sizes and knobs (0 on error); a plan's calls take
 * the arguments of fcfs_forward / fcfs_batch / fcfs_adjoint without the sizes
 * it holds (V may be smaller than the plan's).
 */
enum { FCFS_PLAN_FORWARD = 0, FCFS_PLAN_BATCH = 1, FCFS_PLAN_ADJOINT = 2 };
enum { FCFS_KNOB_FORM = 0, FCFS_KNOB_SPLITS = 1, FCFS_KNOB_PAIR = 2, FCFS_KNOB_UNIT_CHUNKS = 3 };
typedef struct fcfs_plan_s* fcfs_plan;
fcfs_status fcfs_plan_create(fcfs_plan* plan, int32_t kind, int64_t V, int32_t n_clips, int32_t T,
                             int32_t K, int32_t prec);
void fcfs_plan_destroy(fcfs_plan plan);
fcfs_status fcfs_plan_set(fcfs_plan plan, int32_t knob, int64_t value);
int64_t fcfs_plan_get(fcfs_plan plan, int32_t knob);
size_t fcfs_plan_workspace_size(fcfs_plan plan);
fcfs_status fcfs_plan_forward(fcfs_plan plan, const int32_t* x, const int32_t* y, const int8_t* s,
                              int64_t V, uint32_t flags, float* F_out, int64_t* area_out,
                              void* workspace, size_t ws_bytes, void* stream);
fcfs_status fcfs_plan_batch(fcfs_plan plan, const int32_t* x, const int32_t* y, const int8_t* s,
                            const int64_t* offsets, int64_t V_total, float* F_out,
                            int64_t* area_out, void* workspace, size_t ws_bytes, void* stream);
fcfs_status fcfs_plan_adjoint(fcfs_plan plan, const int32_t* x, const int32_t* y, const int8_t* s,
                              int64_t V, const float* dF, float* gx, float* gy,
                              void* workspace, size_t ws_bytes, void* stream);

/*
 * Continuous cosine series of one clip (the cosine extension of FCFS named in
 * the concluding section; the paper gives no formula, so this keeps the
 * conventions of the Fourier block: the inner product with the basis, no
 * basis normalisation, C(0,0) = area):
 *
 *     C(k,l) = integral over the image of cos(pi k x / T) cos(pi l y / T) dx dy,
 *     0 <= k, l <= K.
 *
 * With the same signed quadrants, C = Xc diag(s) Yc^T,
 * Xc[k,v] = integral_{x_v}^T cos(pi k t / T) dt = -(T / (pi k)) sin(pi k x_v / T)
 * (T - x_v at k = 0).  For a balanced corner set this reduces to the exact
 * area at (0,0), the axis lines C(k,0) = (T/(pi k)) sum s y sin(pi k x / T)
 * (exact integer sums, as Eqs. Fk0 and F0l) and
 * C(k,l) = T^2/(pi^2 k l) sum s sin(pi k x / T) sin(pi l y / T): the
 * quarter-plane contraction at period 2T with sine rows only.
 *   x, y, s, V : as for fcfs_forward; coordinates 0 <= x, y <= T.
 *   T          : power of two, 4 <= T <= 32768 (the tables have period 2T).
 *   K          : 1 <= K <= 4096.
 *   prec       : FCFS_PREC_SPLIT_F16 (tensor cores on CTA pairs) or FCFS_PREC_FP32.
 *   flags      : must be 0 (no device validation).
 *   C_out      : (K+1)^2 float32 (device), row-major, C_out[k*(K+1) + l] = C(k,l),
 *                written completely.
 *   area_out   : one int64 (device), the exact area C(0,0).
 *   workspace  : >= fcfs_cosine_workspace_size(V, T, K, prec) bytes, 256-byte aligned.
 * Four kernels; returns FCFS_OK once enqueued.
 */
size_t fcfs_cosine_workspace_size(int64_t V, int32_t T, int32_t K, int32_t prec);
fcfs_status fcfs_cosine(const int32_t* x, const int32_t* y, const int8_t* s, int64_t V,
                        int32_t T, int32_t K, int32_t prec, uint32_t flags,
                        float* C_out, int64_t* area_out,
                        void* workspace, size_t ws_bytes, void* stream);

/*
 * Continuous Haar transform of one clip (Sec. II-C; the PCHT of Sec. III-B
 * computes the same coefficients by a pruned recursion per polygon):
 * coefficients up to level J of the orthonormal 2-D Haar basis of the tile
 * [0,T) x [0,T), as one square of side 2^J (FP64, row-major, first index
 * along x):
 *     W[0][0]               = <f, phi_000>             = area / T
 *     W[2^j + kx][ky]       = <f, psi^(hg)_{j,kx,ky}>  (detail along x)
 *     W[kx][2^j + ky]       = <f, psi^(gh)_{j,kx,ky}>  (detail along y)
 *     W[2^j + kx][2^j + ky] = <f, psi^(hh)_{j,kx,ky}>
 * for 0 <= j < J, 0 <= kx, ky < 2^j.  With A_nm the areas of the image in the
 * four children of the dyadic square (j, kx, ky) (n along x, m along y), the
 * details are (2^j / T)(A00 + A01 - A10 - A11), (2^j / T)(A00 - A01 + A10 - A11)
 * and (2^j / T)(A00 - A01 - A10 + A11).  The areas are exact integers, so every
 * coefficient is exact in FP64.
 *   x, y, s, V : signed corners as for fcfs_forward; 0 <= x, y <= T.
 *   T          : power of two, 4 <= T <= 65536.
 *   J          : 0 <= J <= min(log2 T, 14).
 *   flags      : must be 0.
 *   W_out      : 4^J doubles (device), written completely.
 *   workspace  : >= fcfs_haar_workspace_size(V, T, J) bytes, 256-byte aligned
 *                (the corners grouped by x, the coarse area grids, and either the
 *                column sums of bands of 32 cell rows -- grids of >= 256 cells a
 *                side with cells up to 1024 wide, built band by band on chip --
 *                or the whole grid of 4^J level-J cell areas, 32-bit for cells up
 *                to 1024 wide, else 64-bit).
 * Returns FCFS_OK once enqueued.
 */
size_t fcfs_haar_workspace_size(int64_t V, int32_t T, int32_t J);
fcfs_status fcfs_haar(const int32_t* x, const int32_t* y, const int8_t* s, int64_t V,
                      int32_t T, int32_t J, uint32_t flags, double* W_out,
                      void* workspace, size_t ws_bytes, void* stream);

/*
 * Forward block for callers that cannot allocate device memory (no counterpart
 * in the paper; it exists for such callers).  Some code cannot call cudaMalloc
 * where it needs the transform: a plugin whose host framework owns all device
 * memory, a real-time loop where an allocation would stall the device, a
 * memory-pool callback that must not re-enter the allocator.  This entry point
 * takes the same inputs and outputs as fcfs_forward but no workspace: its
 * scratch is a fixed array of FCFS_NOALLOC_SCRATCH_BYTES compiled into the
 * library, which every GPU that loads the library keeps until the process
 * exits.  Nothing is allocated per call, by the caller or by the library.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 *    The address is looked up again when the device's context has changed
 *    since (for example after cudaDeviceReset, which reloads the module).
 *  - All calls share the array and it keeps the last call's contents (cached
 *    sincos tables; each call zeroes its accumulators itself).  Calls that
 *    overlap on the GPU (other streams, unordered host threads) race: issue
 *    them one after another.
 *  - A clip whose workspace exceeds the array runs with fewer vertex splits;
 *    if even one split does not fit (about K > 1400), FCFS_EUNSUPPORTED.
 *  - flags must be 0 (no device validation).  Device-side status (a bounded
 *    wait that gave up) is read with fcfs_noalloc_status.
 */
#define FCFS_NOALLOC_SCRATCH_BYTES (32u << 20)
fcfs_status fcfs_forward_noalloc(const int32_t* x, const int32_t* y, const int8_t* s, int64_t V,
                                 int32_t T, int32_t K, int32_t prec, uint32_t flags,
                                 float* F_out, int64_t* area_out, void* stream);

/* Status word of the last fcfs_forward_noalloc call on the current device:
 * waits for `stream`, then returns FCFS_ETIMEOUT if a bounded device wait of
 * that call gave up, FCFS_OK otherwise (FCFS_ECUDA if the read fails). */
fcfs_status fcfs_noalloc_status(void* stream);

/*
 * Environment: FCFS_PDL=0 launches the contraction kernel without programmatic
 * dependent launch (no overlap of its set-up with the prep kernel; the work is
 * the same).  FCFS_COOPERATIVE=0 launches fused calls without the cooperative
 * attribute: nothing then guarantees that every CTA is resident, and the grid
 * barrier's bounded wait ends the call with FCFS_ETIMEOUT if one is not (on an
 * otherwise idle GPU they all fit).  Both are for kernel profilers that cannot
 * replay such launches; leave them unset otherwise.
 *
 * Measurement and tuning hooks.  fcfs_profile_enable(1) makes every later call bracket
 * each of its stages with CUDA events on the caller's stream; after a call,
 * fcfs_profile_read() waits for the last event and writes up to n stage
 * durations in milliseconds (0: prep/tables, 1: area and axis lines,
 * 2: contraction, 3: reduce and epilogue).  Returns the number written.
 * In a fused call (below) stages 1 and 3 run inside stage 2 and read 0.
 * fcfs_debug_set_splits(n) forces n vertex splits (0: automatic choice).
 * fcfs_debug_set_fuse(0) makes fcfs_forward keep the axis-line DFT and the
 * split-K reduction in kernels of their own; 1 (the default) lets the
 * split-FP16 path run them inside the contraction kernel whenever its CTAs fit
 * on the GPU at once (one cooperative launch; the results are the same up to
 * FP32 rounding order, which is fixed either way).
 * Not thread-safe; meant for benchmarks and tests.
 */
void fcfs_profile_enable(int32_t on);
int32_t fcfs_profile_read(float* ms, int32_t n);
/* Kernel timing by stage name: fcfs_kernel_timing_enable(1) clears the records
 * and makes every later call bracket each of its stages (a kernel, or a short
 * group such as the three grouping kernels) with two events on the caller's
 * stream, up to 64 records; (0) stops recording.  fcfs_kernel_timing_count()
 * waits for the last record and returns how many there are; name(i) and ms(i)
 * give stage i's name (a static string) and its elapsed time (-1 on error).
 * Events between launches serialise stages that would otherwise overlap: use
 * it for measurement passes, not for timed runs. */
void fcfs_kernel_timing_enable(int32_t on);
int32_t fcfs_kernel_timing_count(void);
const char* fcfs_kernel_timing_name(int32_t i);
float fcfs_kernel_timing_ms(int32_t i);
void fcfs_debug_set_splits(int32_t n);
void fcfs_debug_set_fuse(int32_t on);
/* Which form fcfs_forward (flags 0) will take for these sizes: 0 the
 * contraction over the V corners, 1 the corners grouped by y and the
 * split-FP16 contraction over the T + 1 values of y, 2 the corners grouped by
 * y and the pruned FFT along y (Step 4's sparse-image DFT with its output
 * limited to |l| <= K, FP32), -1 for unsupported sizes.  The automatic choice
 * (fcfs_debug_set_hybrid(1), the default) compares cost estimates of the
 * forms the call may take; fcfs_debug_set_hybrid(0), (2) and (3) force the
 * first, second and third. */
int32_t fcfs_forward_grouped(int64_t V, int32_t T, int32_t K, int32_t prec);
/* The same for fcfs_adjoint: 0 the contraction per corner (tensor cores, or
 * the plain FP32 kernel), 1 the corners grouped by y (gx) and by x (gy) and
 * the split-FP16 contraction over the T + 1 values of the grouped coordinate
 * (split-FP16 calls only), 2 grouped with the pruned FFT along it (the
 * adjoint's sums over b as input-pruned FFTs, then one dot per corner; FP32,
 * any precision, 16 <= T, 2K <= min(T, 4096)); -1 for unsupported sizes or
 * precision.  The automatic choice compares cost estimates of the forms;
 * fcfs_debug_set_hybrid(0), (2) and (3) force the first, second and third
 * where they apply. */
int32_t fcfs_adjoint_grouped(int64_t V, int32_t T, int32_t K, int32_t prec);
/* fcfs_debug_set_pair(0) keeps single-clip split-FP16 calls on one-CTA
 * 128 x 256 tiles; 1 (the default) runs clips with 2K >= 256 on CTA pairs
 * (2-SM MMA on 256 x 256 tiles).  Must not change between fcfs_workspace_size
 * and the call that uses the workspace. */
void fcfs_debug_set_pair(int32_t on);
/* Failure-detection test hook: with n > 0 the grid barrier of later fused
 * calls waits for n more CTAs than were launched.  Its wait is bounded (about
 * a second of SM clock), so the call ends with the status FCFS_ETIMEOUT
 * (fcfs_get_status) and an unwritten block, and the context stays usable.
 * 0 (the default) restores normal calls. */
void fcfs_debug_set_barrier_extra(int32_t n);
/* Row-binned contraction of single-clip split-FP16 calls on CTA pairs (the
 * corners grouped by y, the off-axis block contracted over the T + 1 values of
 * y instead of the V corners; the binning of Steps 2-3 carried into Step 4):
 * mode 0 never, 1 (the default) when a cost estimate of the forms favours
 * it (fcfs_forward_grouped tells), 2 the split-FP16 contraction over y whenever
 * the call is eligible (split FP16, 2K >= 256, no device validation), 3 the
 * pruned FFT along y whenever eligible (any precision, K <= 4096, no device
 * validation).  Batches group when
 * V >= 8 n (T + 1) and K >= 256.  The adjoint takes its forms under the same
 * modes (0 per corner, 2 grouped contraction, 3 grouped pruned FFT, 1 the
 * cheapest estimate; fcfs_adjoint_grouped tells).  Same results within
 * the split-FP16 error bound.  Must not change between fcfs_workspace_size and
 * the call that uses the workspace. */
void fcfs_debug_set_hybrid(int32_t mode);
/* Stages of a call that do not depend on its main sequence (the axis lines of
 * the grouped forward forms, the grouping of the pruned-FFT adjoint) run on a
 * second stream of the calling thread, forked from and joined back into the
 * call's stream by events (graph-capturable): on = 1, the default unless the
 * environment has FCFS_OVERLAP=0.  With 0 every stage runs on the call's
 * stream, in order, which is what per-stage timing (fcfs_kernel_timing_*)
 * needs to see each stage alone.  Same results either way. */
void fcfs_debug_set_overlap(int32_t on);

/* Vertex-split granularity of fcfs_batch: n pipeline chunks (64 corners on the
 * tensor path, 32 on the FP32 path) per unit; 0 restores the default of 4096
 * corners.  Process-wide; the autotuner sets it per workload. */
void fcfs_set_batch_unit_chunks(int32_t n);

/*
 * Synchronise `stream` and return the device status word of the last call that
 * used `workspace` (FCFS_OK, FCFS_EINVAL_DATA or FCFS_ETIMEOUT).
 */
fcfs_status fcfs_get_status(const void* workspace, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FCFS_H */
