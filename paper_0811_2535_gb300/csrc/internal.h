// Internal interfaces between the plan (moa_fft.cu), the pass kernels
// (pass_kernels.cu) and the twiddle generator (twiddle.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace moa {

enum PassKind {
    PASS_ROW = 0,
    PASS_COL = 1,
    PASS_TC = 2,
    PASS_LIFT3 = 3,  // fused second and third pass of a three-level lift (lift3.cu);
                     // logF = log2 cA, logN = log2 cB
    PASS_PLANE1 = 4, // 3-D 256^3, first of two passes: axis 2 and the first radix-16 step of
                     // axis 1 (pass_kernels.cu); O = number of arrays
    PASS_PLANE2 = 5  // 3-D 256^3, second pass: the rest of axis 1 and axis 0 (pipe_kernels.cu)
};

enum PassFlags {
    FLAG_CONJ_IN = 1,    // conjugate on load (sign +1 via conj(F_-(conj x)))
    FLAG_CONJ_OUT = 2,   // conjugate on store
    FLAG_TW4 = 4,        // multiply column outputs by w_{N*C}^(k*i) (four-step twiddle)
    FLAG_PDL = 8,        // launch as a programmatic dependent launch of the previous kernel in the
                         // stream (the row, column and pipelined pass kernels wait for it on the device)
    FLAG_SHORT_WAIT = 16 // fault injection for tests: the pipelined kernels give up on a tile load
                         // that has not landed at its first test (MOA_ERR_TIMEOUT, no GPU fault)
};

// Transforms per tile that a plan gives a column pass of 2^logN points over
// C columns, and a row pass over O rows (transposed: its store is the
// four-step transpose), for tiles of 2^tile points (10..14; anything else:
// the default, 2^12 or MOA_TILE_LOG2); the allocation-free entry point uses
// the same.
int pick_logF_col(int logN, int64_t C, int tile = -1);
int pick_logF_row(int logN, int64_t O, bool transposed, int tile = -1);

// One kernel launch: N-point transforms (N = 2^logN <= 4096) along one axis.
//  PASS_COL: view [O][N][C] (row-major), transform along the middle axis,
//            F consecutive columns per tile, output in the same view; with
//            Rt > 1 (a lifted axis, second half) output row k of o goes to
//            row (o % Rt) + Rt*k of the [O/Rt][N*Rt][C] view.  The four-step
//            twiddle (tw4) is w_M^((col / cdiv) * row), row the output row in
//            that view and M = N * Rt * C / cdiv: with cdiv = 1, Rt = 1 the
//            twiddle w_n^(j2*k1) of the lifted 1-D transform; with cdiv = the
//            inner extent, the twiddle between the two halves of an axis
//            lifted inside a multi-D array.
//  PASS_ROW: view [O][N], transform along contiguous rows, F rows per tile;
//            output row o, index k goes to (o / Rt)*(N*Rt) + (o % Rt) + Rt*k
//            (Rt = 1: natural order; Rt = r: the four-step transpose).
struct PassDesc {
    int kind;
    int logN;
    int64_t O;
    int64_t C;      // PASS_COL only
    int64_t Rt;     // PASS_ROW only
    int logF;       // log2 of transforms per tile
    int src, dst;   // buffer ids: 0 = user in, 1 = user out, 2 = workspace
    int tw4;        // apply the four-step twiddle (PASS_COL)
    int pipe;       // 1: persistent TMA-pipelined kernel (pipe_kernels.cu)
    int blk;        // blocked workspace of the lifted transform (pipe kernels only):
                    // 1 = pass 1 writes 4 x 4 blocks, 2 = pass 2 reads them
    int umma;       // PASS_TC: 1 = tcgen05 kernel (tc_umma.cu), 0 = mma.sync kernel
    int cdiv;       // PASS_COL twiddle: column divisor (0 or 1: none)
    int twlog;      // PASS_COL twiddle: log2 M of its table (0: the plan's main table lo/hi)
    int sched;      // generic row and column passes: radix schedule V of Sched<logN, V> (0, 1, 2),
                    // or 3 = row_warp_kernel (natural-order rows of 128..512 points, cross-lane
                    // stages by warp shuffles)
};

struct TwiddleSet {
    const float2 *stage[13];   // per logN: stage tables (Sched<logN> layout), or null
    const float2 *vstage[4][13];   // per schedule V = 1, 2 and logN: stage tables of Sched<logN, V>;
                                   // vstage[3]: row_warp_kernel's tables (V = 0 uses `stage`)
    const float2 *lo, *hi;     // two-level table of w_n^e: lo[e & (2^h-1)] * hi[e >> h]
    int h;
    const float2 *xlo[32], *xhi[32];   // further two-level tables of w_M, by log2 M (lifted axes)
    int xh[32];
    const float2 *tc;          // tensor-core path: per-stage full tables
};

// Launch one pass.  `flags` carries FLAG_CONJ_*; FLAG_TW4 is derived from d.
// `status` is the plan's device status word (bounded waits report there).
cudaError_t launch_pass(const PassDesc &d, const float2 *in, float2 *out, const TwiddleSet &tw,
                        int flags, cudaStream_t stream, int *status);
// The pipelined strided kernels (N = 1024..4096, four transforms per tile):
// usable when the driver exposes cuTensorMapEncodeTiled.  The input must be
// 16-byte aligned.
bool pipe_supported();
// whether the pipelined column passes of N = 4096 run two columns per thread
// (pipe_col2_kernel; MOA_COL2=0 selects the four-column pipe_col_kernel)
bool pipe_col2_active();
// Tiled TMA tensor map of 8-byte elements (complex64 moved as 64-bit words):
// dims / box in elements, innermost first; strides in bytes of dims 1..rank-1.
bool encode_c64_map(CUtensorMap *map, const void *base, int rank, const uint64_t *dims, const uint64_t *strides,
                    const uint32_t *box);
cudaError_t prepare_pipe_kernels();
cudaError_t launch_pipe_pass(const PassDesc &d, const float2 *in, float2 *out, const TwiddleSet &tw, int flags,
                             cudaStream_t stream, int *status);
// The two passes of the two-pass 3-D transform of d.O arrays of 256^3: in ->
// ws (w256[e] = w_256^e, e < 256), then ws -> out (ws 16-byte aligned).
cudaError_t launch_plane1(const PassDesc &d, const float2 *in, float2 *ws, const TwiddleSet &tw, const float2 *w256,
                          int flags, cudaStream_t stream);
cudaError_t launch_pipe_plane2(const PassDesc &d, const float2 *in, float2 *out, const TwiddleSet &tw, int flags,
                               cudaStream_t stream, int *status);
// Tensor-core rows (tc_kernels.cu): 1-D transforms of N = 256 or 4096 along
// contiguous rows, radix-16 blocks as FP16 (hi/lo) or BF16 (hi/mid/lo) GEMMs.
// `tw` holds the per-stage tables w_M^(u*k), k < 16 (tc_table_entries).
int tc_table_entries(int logN);
cudaError_t launch_tc_pass(const PassDesc &d, bool bf16, const float2 *in, float2 *out, const float2 *tw, int flags,
                           cudaStream_t stream);
// dst[k*M1 + u] = w_M^(u*k mod M), k < 16, u < M1 (sign -1).
// The same pass on the tcgen05 tensor cores (operands in shared memory,
// accumulators in tensor memory); `status` receives MOA_ERR_TIMEOUT if a
// wait for the products gives up.
cudaError_t launch_umma_pass(const PassDesc &d, bool bf16, const float2 *in, float2 *out, const float2 *tw, int flags,
                             cudaStream_t stream, int *status);
// Fused second and third pass of a three-level lifted 1-D transform of
// n = r * cA * cB points (lift3.cu).  The queue is implicit (the middle
// tiles of unit u, then `lag` units later the last tiles of unit u);
// `ticket` is followed by two counters per unit (middle tiles finished, last
// tiles that have read the unit); `ring` holds `ring_units` units of the
// intermediate, unit u in slot u % ring_units.
struct Lift3Launch {
    // TMA tensor maps in device global memory: the workspace as
    // [B r cA rows][cB] (box 4096/cA x cA) and the ring as
    // [ring rows][cA][cB] (box cB x 1 x 4096/cB)
    const CUtensorMap *map_mid, *map_last;
    int lag;
    int *ticket;
    float2 *ring;
    int ring_units;
    int nunits;
    int grid;
    const float2 *lo, *hi;   // two-level table of w_c^e, c = cA * cB
    int h;
    int loga, logb, logr;
    int middle_per_unit;     // middle-pass tiles per unit (= cA)
    int ex_entries;          // exchange buffer entries (complex64) in shared memory
    size_t smem_bytes;       // dynamic shared memory per block
};
int lift3_blocks_per_sm();
cudaError_t launch_lift3(const Lift3Launch &l, float2 *out, const float2 *stage_a, const float2 *stage_b, int flags,
                         cudaStream_t stream, int *status);
cudaError_t generate_full_stage(float2 *dst, int64_t M, int64_t M1, cudaStream_t stream);
// Shared memory bytes and threads per block of a pass.
size_t pass_smem_bytes(const PassDesc &d);
int pass_threads(const PassDesc &d);
// One-time per-process kernel attribute set-up (dynamic shared memory).
cudaError_t prepare_kernels();

// Twiddle generation (FP64 on the device, rounded once to FP32).  Stage
// tables of schedule V (0, 1, 2: Sched<logN, V>; 3: the warp-shuffle row
// kernel, rows k = 1, 2, 3, 4, 8, 12 of w_N^(u*k), u < N/16, then w_{N/16}^u);
// -1 entries for a schedule that does not exist for logN.
int stage_table_entries(int logN, int V = 0);
cudaError_t generate_stage_table(float2 *dst, int logN, cudaStream_t stream, int V = 0);
// whether schedule V (0..3) exists for 2^logN points
bool sched_exists(int logN, int V);
// w_n^e for e < 2^h (lo) and w_n^(e*2^h) for e < n/2^h (hi); sign -1.
cudaError_t generate_two_level(float2 *lo, float2 *hi, int logn, int h, cudaStream_t stream);

}  // namespace moa
