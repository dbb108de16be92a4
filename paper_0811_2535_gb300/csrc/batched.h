// Work-queue types of the batched persistent launch (batched.cu) shared
// with the plan (moa_fft.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace moa {

// One queue entry.
//   kind 0 (small): `count` transforms of length 2^logn whose offsets are
//                   offs[first .. first+count-1], all in one block.
//   kind 1 (column tile) / kind 2 (row tile): tile `tile` of the column or
//                   row phase of the single transform offs[first], of length
//                   2^logn lifted as 2^logr x 2^(logn-logr).  A row tile
//                   starts once counter[first] shows that all 2^logn / 4096
//                   column tiles of its transform are done.
struct BatchTask {
    int32_t first;
    int16_t count;
    int16_t tile;
    int8_t logn;
    int8_t logr;
    int8_t kind;
    int8_t pad;
};

struct BatchTables {
    const float2 *stage[13];   // per-length stage tables (Sched layout)
    const float2 *lo[17];      // two-level tables of w_n^e for large n (indexed by log n)
    const float2 *hi[17];
    int h[17];
};

struct BatchLaunch {
    const BatchTask *tasks;
    int ntasks;
    int *ticket;               // ticket, then one completion counter per transform (cleared per exec)
    int ncounters;
    const int64_t *offs;       // element offset of each transform, in queue order
    float2 *ws;                // workspace mirroring the input layout (large tasks)
    const BatchTables *tables;   // device copy of the table pointers
    unsigned grid;
    // Bounded waits of the row tiles: at most max_polls polls of the counter.
    // Fault injection for tests (MOA_FAULT_WAIT=1 at plan time): wait_extra = 1
    // makes every row tile wait for one column tile more than its transform
    // has, a count nothing reaches, so each wait runs out and reports
    // MOA_ERR_TIMEOUT (the tile is skipped; nothing hangs or faults).
    int max_polls;
    int wait_extra;
};

int batched_blocks_per_sm();
cudaError_t launch_batched(const BatchLaunch &b, const float2 *in, float2 *out, int flags, cudaStream_t stream,
                           int *status);

}  // namespace moa
