// sl_fused.cuh -- work maps of the fused (batched) launches.
//
// A batch of replicas can step with ONE launch per kernel of the step: the launch is a
// persistent grid whose blocks walk a device-side table of work items.  Work item w belongs
// to slot r when w0[r] <= w < w0[r + 1] (a prefix over the slots' own block counts, in
// device memory and rewritten at the start of every step, so replicas join, leave or finish
// without a new graph capture; an idle slot adds no blocks); the slot's argument block sits
// at index r of a device array, and the item is that replica's local block w - w0[r] of
// w0[r + 1] - w0[r].  Every kernel of the step is written as a device body over (arguments,
// local block, local block count), called by the single-system kernel with (its arguments,
// blockIdx.x, gridDim.x) and by the fused kernel for every work item.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace sl {

struct WorkMap {
    const int64_t *w0;   // [nrep + 1] prefix of the slots' block counts (device)
    int nrep;            // number of slots
};

// the tensor-core network's arguments for one replica (the TMA map read from global memory;
// the map type carries its own alignment of at least 64 bytes)
struct MlpArgs {
    CUtensorMap qmap;    // descriptors [DIM] rows x n atoms, 128 x 66 boxes
    int64_t n;
    float *fp, *ei;
    int *status;
    const int *skip;     // non-null: the slot's tiles are passed over while *skip
    const void *wimg;    // the weights' FP16 hi/lo operand images (20,480 bytes, 16-byte aligned)
};
static_assert(alignof(CUtensorMap) >= 64, "tensor maps are 64-byte aligned");

// the CUDA-core network's arguments for one replica
template <typename R>
struct NetArgs {
    const R *q;
    R *fp, *ei;
    int64_t n, qs;
    const int *skip;     // non-null: the slot's atoms are passed over while *skip
};

// the slot of work item w: the last slot r with w0[r] <= w (idle slots before it have
// w0[r] == w0[r + 1] and are passed over)
__device__ __forceinline__ int work_replica(const WorkMap &m, int64_t w) {
    int lo = 0, hi = m.nrep - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(m.w0 + mid) <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The argument block of slot r in shared memory: the block copies it when it moves to another
// slot (block-uniform).  A body then reads its arguments from shared memory, which the global
// stores it makes cannot alias, so the compiler keeps them out of its loops.
template <typename A>
__device__ __forceinline__ const A &slot_args(const A *__restrict__ tab, int r, int &cur) {
    __shared__ __align__(16) uint32_t s_args[(sizeof(A) + 3) / 4];
    static_assert(sizeof(A) % 4 == 0, "argument blocks are whole words");
    if (r != cur) {
        __syncthreads();   // every thread is done with the previous slot's arguments
        const uint32_t *src = reinterpret_cast<const uint32_t *>(tab + r);
        for (int k = threadIdx.x; k < (int)(sizeof(A) / 4); k += blockDim.x) s_args[k] = __ldg(src + k);
        __syncthreads();
        cur = r;
    }
    return *reinterpret_cast<const A *>(s_args);
}

// body(args of the item's slot, local block, local block count) for every work item of the
// map, the block's items in turn (block-uniform, so bodies may synchronise the block)
template <typename A, typename Body>
__device__ __forceinline__ void for_each_work(const A *__restrict__ tab, const WorkMap &m, Body body) {
    const int64_t total = __ldg(m.w0 + m.nrep);
    int cur = -1;
    for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
        const int r = work_replica(m, w);
        const int64_t b0 = __ldg(m.w0 + r);
        body(slot_args(tab, r, cur), w - b0, __ldg(m.w0 + r + 1) - b0);
        __syncwarp();
    }
}

// Where the one-item-per-block kernels find their block's slot.  A batch launch (tab non-null)
// covers every occupied slot in a fixed layout: block w belongs to slot item_slot[w] (-1: no
// slot) as its local block w - start[slot]; the slot takes part in this step when its range in
// the step's work map m is non-empty.  A system's own launch (tab null) has one slot, whose
// arguments come as a kernel parameter, and block w is its local block w.
struct SlotMap {
    const int *item_slot;
    const int64_t *start;
    WorkMap m;
};

// body(args, local block, 0) for the block's work item: the arguments are copied into shared
// memory first (from the kernel parameter or from the table), so the body is the same compiled
// code for both kinds of launch.  The hot kernels take this form: one item per block, no loop,
// whose state would stay live across the body and cost registers.
template <typename A, typename Body>
__device__ __forceinline__ void one_work(const A *__restrict__ tab, const SlotMap &sm, const A &solo, Body body) {
    __shared__ __align__(16) uint32_t s_args[sizeof(A) / 4];
    static_assert(sizeof(A) % 4 == 0, "argument blocks are whole words");
    int64_t blk = blockIdx.x;
    const uint32_t *src = reinterpret_cast<const uint32_t *>(&solo);
    if (tab) {   // uniform across the grid
        const int r = __ldg(sm.item_slot + blockIdx.x);
        if (r < 0) return;
        const int64_t a0 = __ldg(sm.m.w0 + r), a1 = __ldg(sm.m.w0 + r + 1);
        blk -= __ldg(sm.start + r);
        if (a1 <= a0) return;   // the slot takes no part in this step
        src = reinterpret_cast<const uint32_t *>(tab + r);
    }
    for (int k = threadIdx.x; k < (int)(sizeof(A) / 4); k += blockDim.x) s_args[k] = src[k];
    __syncthreads();
    body(*reinterpret_cast<const A *>(s_args), blk, 0);
}

// body(args of the item's slot, local block, local block count) for work item blockIdx.x of
// the map alone: one item per block (blocks past the map's total return at once), without the
// loop's state living across the body.
template <typename A, typename Body>
__device__ __forceinline__ void map_item(const A *__restrict__ tab, const WorkMap &m, Body body) {
    const int64_t w = blockIdx.x;
    if (w >= __ldg(m.w0 + m.nrep)) return;   // block-uniform
    const int r = work_replica(m, w);
    const int64_t b0 = __ldg(m.w0 + r);
    int cur = -1;
    body(slot_args(tab, r, cur), w - b0, __ldg(m.w0 + r + 1) - b0);
}

// The same as for_each_work, passing over every item of a slot for which idle(args) holds (block-uniform:
// the block moves on to its first item past the slot's range).
template <typename A, typename Idle, typename Body>
__device__ __forceinline__ void for_each_work_unless(const A *__restrict__ tab, const WorkMap &m, Idle idle,
                                                     Body body) {
    const int64_t total = __ldg(m.w0 + m.nrep);
    int cur = -1;
    for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
        const int r = work_replica(m, w);
        const int64_t b0 = __ldg(m.w0 + r), b1 = __ldg(m.w0 + r + 1);
        if (idle(tab[r])) {
            w += (b1 - 1 - w) / gridDim.x * gridDim.x;   // this block's last item of slot r
            continue;
        }
        body(slot_args(tab, r, cur), w - b0, b1 - b0);
        __syncwarp();
    }
}

}  // namespace sl
