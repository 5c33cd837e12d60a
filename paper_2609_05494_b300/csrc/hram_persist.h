// hram_persist.h -- internal interface between the C-ABI (hram_capi.cu) and
// the persistent batched kernel (hram_persist.cu).
#pragma once
#include <cuda_runtime.h>

namespace hr {
struct Consts;
struct Bufs;

// Resident 256-thread blocks of the persistent kernel per multiprocessor.
int persist_blocks_per_sm(int closure);

// One cooperative launch of nblk blocks: blk[b] = (case, rank in the case),
// case_nblk[c] = blocks of case c, bar = 2 ints per case (zeroed), err = one
// int (zeroed).  Runs up to max_steps steps of every case (until each is
// done).  Returns 0, or -1 when the launch is refused.
int persist_launch(const Consts *dK, const Bufs *dB, const int2 *blk, const int *case_nblk, int nblk,
                   int *bar, long long spin_limit, long long max_steps, int *err, int closure,
                   cudaStream_t s);
}  // namespace hr
