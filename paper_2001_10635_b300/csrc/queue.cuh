// queue.cuh -- records shared by the host side of the device work queue
// (queue.cu) and its persistent kernel (onchip_kernels.cuh).
//
// The queue serves MM / CGB queries small enough for one block (2n <= QMAX x
// 512 components) while other work runs on the GPU: the host appends each
// query to a ring in mapped page-locked memory and publishes it by advancing
// the ring's tail; the blocks of a persistent kernel claim published items
// one at a time, integrate the whole horizon in shared memory, write the box
// and raise the item's done word.  A block that finds no work for the idle
// limit leaves, so an idle queue holds no SM.
#pragma once

#include "onchip.cuh"

namespace reach {

constexpr int QUEUE_THREADS = 512;
constexpr int64_t QUEUE_MAX_COMPONENTS = (int64_t)QMAX * QUEUE_THREADS;   // 2n of the largest item
static_assert(QUEUE_MAX_COMPONENTS == 2 * REACH_QUEUE_MAX_N, "the public size limit is one block's items");

// one published query (written by the host before the tail passes it)
struct QueueItem {
    OnItem it;         // it.status is ignored: the kernel uses the slot's device word
    int64_t ticket;
};

// how a block of the persistent kernel left (its per-block exit word)
enum : int { QEXIT_RUNNING = 0, QEXIT_IDLE = 1, QEXIT_STOPPED = 2 };

struct QueueArgs {
    const QueueItem *ring;            // mapped: cap items
    const long long *tail;            // mapped: items published so far
    const int *stop;                  // mapped: nonzero asks idle blocks to leave at once
    long long *done;                  // mapped: done[slot] = ticket once the slot's results are visible
    int *hstatus;                     // mapped: the slot item's status bits (ST_*)
    int *exited;                      // mapped: one exit word per block of this launch
    unsigned long long *head;         // device: next item to claim
    int *dstatus;                     // device: per-slot status bits while the item runs
    int cap;
    unsigned long long idle_ns;       // a block leaves after this long without an item
};

}  // namespace reach
