// sl_batch.h -- argument tables of the step's kernels (not part of the ABI).
//
// Every kernel of a step (first half, rebuild group, radial, angular, network, backward,
// second half) reads its arguments from a device table of per-slot argument blocks and walks
// a work map (sl_fused.cuh).  A batch keeps one slot per replica and launches each kernel once
// over all of them (persistent grids; the work maps are rebuilt at the start of every step by
// a one-block plan kernel from per-slot budgets of steps left, so replicas with different
// step counts share the launches until each budget is spent, and the captured graphs survive
// admissions and retirements).  A system stepping alone launches the same kernels over a table
// of its own, whose slots are its launch variants (kinds below).  So a replica's arithmetic is
// the same compiled code alone and in a batch, and its results are bit-identical; a slot's
// block count per kernel is the one a single launch of its shape would have.
#pragma once

#include <cstring>
#include <vector>

#include "sl_internal.h"
#include "sl_fused.cuh"

namespace sl {

// kernels of one step, in launch order
enum FusedKernel {
    FK_FIRST, FK_BIN, FK_SCAN, FK_SCATTER, FK_CELLSORT, FK_LISTS, FK_REV, FK_FINISH,
    FK_CRAD, FK_ANG, FK_NET, FK_BWD, FK_SECOND, FK_N
};
constexpr int FUSED_LAUNCHES_PER_STEP = 1 + FK_N + 1;   // plan, the kernels, the flag clear
constexpr int FUSED_MAX_SLOTS = 4096;
// atoms-per-block classes of the kernels that take one work item per block: the halves (256
// atoms), the radial kernel and the FP64 network (128), the angular and backward kernels (a
// quad block's atoms)
enum { IC_HALF = 0, IC_ATOM = 1, IC_QUAD = 2, IC_N = 3 };

// what a slot's entries are set up for
enum SlotKind {
    SK_STEP = 0,   // a step: conditional rebuild; evaluation at the state, no virial
    SK_FULL = 1,   // unconditional rebuild; evaluation at the state with the virial parts
    SK_MID = 2,    // evaluation at the midpoint point (midpoint iteration), with its skip flag
    SK_N = 3
};

// tables of `cap` slots, each array cap entries long: the host image and the device copy
// share this layout
struct FusedTables {
    int prec = 0, cap = 0;
    // byte offsets of the arrays in the image
    size_t o_blocks = 0;   // int64 [FK_N][cap]: each slot's block count per kernel
    size_t o_left = 0;     // int64 [cap]: steps left (set per call, counted down by the plan kernel)
    size_t o_first = 0, o_second = 0, o_bin = 0, o_lists = 0, o_rev = 0, o_eval = 0, o_net = 0;
    size_t o_w0 = 0;       // int64 [FK_N][cap + 1]: the current step's work maps (batches)
    size_t upload_bytes = 0;   // the host-written part: [0, upload_bytes)
    size_t bytes = 0;
    unsigned char *dev = nullptr;   // device base
    unsigned grid[FK_N] = {};       // grid of each kernel (batches)

    template <typename T>
    const T *at(size_t off) const { return reinterpret_cast<const T *>(dev + off); }
    WorkMap map(int k) const {
        return WorkMap{reinterpret_cast<const int64_t *>(dev + o_w0) + (size_t)k * (cap + 1), cap};
    }
};
// the layout of tables of `cap` slots (offsets and sizes; no memory)
void fused_layout(FusedTables &t, int prec, int cap);

// One launch: the work map (the loops of the rebuild group and the network; in a batch also
// each slot's part in the step), the block -> slot layout of a batch's one-item-per-block
// kernels, or, for a system's own launch of those kernels and of the network, its argument
// block (a host copy, passed as a kernel parameter); grid, threads per block (0: the kernel's
// default) and register-budget variant (0: default).
struct Launch {
    WorkMap m;
    const int *item_slot = nullptr;
    const int64_t *start = nullptr;
    const void *solo = nullptr;
    const int *quick = nullptr;   // a system's own conditional rebuild: its flag (see sl_neighbors.cu)
    unsigned grid = 0;
    int block = 0;
    int minb = 0;
    SlotMap slots() const { return SlotMap{item_slot, start, m}; }
};

// the kernel parameter of a launch: the system's own argument block, or zeros (a batch's)
template <typename A>
A solo_args(const Launch &L) {
    A a;
    if (L.solo) std::memcpy(&a, L.solo, sizeof(A));
    else std::memset(&a, 0, sizeof(A));
    return a;
}

// sizes of the per-slot argument blocks (sl_integrate.cu, sl_eval2.cu, sl_nep.cu)
void fused_half_sizes(int prec, size_t *first, size_t *second);
size_t fused_eval_size(int prec);
size_t fused_net_size(int prec);

// Each writes slot r's argument blocks of its kernels, set up for `kind`, into the host
// image, and the slot's block count of each of its kernels (default shapes) into blocks[k].
void fused_put_half(Sys &s, int r, const FusedTables &t, unsigned char *img, int64_t *blocks);
void fused_put_rebuild(Sys &s, int r, int kind, const FusedTables &t, unsigned char *img, int64_t *blocks);
void fused_put_eval(Sys &s, int r, int kind, const FusedTables &t, unsigned char *img, int64_t *blocks);
void fused_put_net(Sys &s, int r, int kind, const FusedTables &t, unsigned char *img, int64_t *blocks);

// persistent grids of the rebuild group and of the tensor-core network (device attributes and
// occupancy); the other kernels take one work item per block (FusedBatch::reserve)
void fused_grids_rebuild(FusedTables &t);
void fused_grid_net(FusedTables &t);

// launches over a table
void launch_fused_plan(const FusedTables &t, cudaStream_t st);
void launch_first_half_t(const FusedTables &t, const Launch &L, cudaStream_t st);
void launch_second_half_t(const FusedTables &t, const Launch &L, bool spin, cudaStream_t st);
// the rebuild group: L[0 .. 5] for the binning, scan, scatter, lists, reverse slots and finish
// kernels; clear: then the flags of the conditional slots in L[0]'s map are cleared; loop: the
// persistent form (a batch's), else one work item per block (a system's own launches)
void launch_rebuild_t(const FusedTables &t, const Launch *L, bool clear, bool loop, cudaStream_t st);
// radial, angular, network, backward; ev (optional, 6 events): recorded before the radial
// kernel, after it, after the angular kernel, after the network and after the backward
template <typename R>
void launch_eval_t(const FusedTables &t, const NepDev<R> &P, const Launch *L /* crad, ang, net, bwd */,
                   cudaStream_t st, cudaEvent_t *ev);
void launch_net_t_tc(const FusedTables &t, const NepDev<float> &P, const Launch &L, cudaStream_t st);
void launch_net_t_fp64(const FusedTables &t, const NepDev<double> &P, const Launch &L, cudaStream_t st);

// The fused step of one batch: its tables (device, and a pinned host image of the
// host-written part), its slots' systems, and two captured graphs over the tables (g steps
// and one step) with the model parameters every system of the batch shares.
class FusedBatch {
public:
    FusedBatch() = default;
    FusedBatch(const FusedBatch &) = delete;
    FusedBatch &operator=(const FusedBatch &) = delete;
    ~FusedBatch();

    // tables for `cap` slots in precision `prec` on the current device; false on failure
    bool setup(int prec, int cap, int device);
    bool ready(int prec, int cap, int device) const {
        return t.dev && t.prec == prec && t.cap == cap && dev_ == device;
    }
    // slot r holds s (null: empty); its entries are rewritten at the next upload whenever the
    // system (told apart by its unique id, not its address) or its capture version changed
    void assign(int r, Sys *s);
    // graphs of g steps and of one step for the model of system m (captured again only when
    // g or the model changes); false on failure
    bool graphs(int g, const Sys &m, cudaStream_t st);
    bool same_model(const Sys &s) const;
    int device() const { return dev_; }
    // the slots' step budgets (and the tables, where an entry changed) to the device, on st
    cudaError_t upload(const int64_t *left, cudaStream_t st);
    // block -> slot layouts for up to `atoms` atoms over all slots: one block per
    // atoms-per-block of the capacity plus one partial block per slot for each kernel that
    // takes one work item per block.  The capacity only grows (to a power of two); growing
    // drops the graphs.  Those kernels' grids cover the occupied slots' blocks only (upload
    // resizes them in the captured graphs), so a capacity above the resident atoms launches
    // no idle blocks.  False when the layout cannot be allocated.
    bool reserve(int64_t atoms);
    int64_t atom_capacity() const { return atom_cap; }
    // one step of every slot with a budget left, queued on st
    void enqueue(cudaStream_t st) const;

    FusedTables t;
    cudaGraphExec_t graph_g = nullptr, graph_1 = nullptr;
    int g = 0;
    int64_t captures = 0;

private:
    void release_graphs();
    void release_items();
    void release();
    // the kernel nodes of the one-item-per-block kernels in the graph just captured (with its
    // executable graph); false when they cannot all be told apart
    bool find_item_nodes(cudaGraph_t graph, cudaGraphExec_t exec, int steps);
    // those nodes' grids set to grid_items in the executable graphs; false on failure
    bool resize_item_nodes();
    int dev_ = -1;
    // grid of each one-item-per-block class in the launches and captured graphs: the occupied
    // slots' blocks of the current layout (follow), else the capacity's blocks (when the
    // captured nodes could not be found)
    int64_t grid_items[IC_N] = {};
    bool follow = true;
    struct ItemNode {
        cudaGraphExec_t exec;
        cudaGraphNode_t node;   // in tmpl[...], which stays alive with the executable graph
        int cls;
    };
    std::vector<ItemNode> item_nodes;
    cudaGraph_t tmpl[2] = {};
    int64_t atom_cap = 0;
    // block -> slot layout per atoms-per-block class (device; pinned host copy), and each
    // slot's first block per class
    int *items = nullptr, *h_items = nullptr;
    int64_t *starts = nullptr, *h_starts = nullptr;
    int64_t item_off[IC_N] = {}, item_cap[IC_N] = {};
    size_t item_bytes = 0;
    bool layout_dirty = true;
    unsigned char *img = nullptr;   // pinned host image of [0, t.upload_bytes)
    std::vector<Sys *> slot;
    std::vector<uint64_t> uid;       // unique id of each slot's system when its entries were written (0: none)
    std::vector<uint64_t> version;
    std::vector<char> stale;
    bool dirty = true;
    bool have_model = false;
    NepDev<double> pd;
    NepDev<float> pf;
};


// A system's own table: slot k set up for kind k, and for every kernel, kind and shape (0: the
// default threads per block, 1: half of them) a work map covering that slot's blocks only.
struct SoloTables {
    FusedTables t;
    std::vector<unsigned char> host;  // host copy of the table (the kernel parameters of its launches)
    int64_t *w0 = nullptr;            // device [FK_N][SK_N][2][SK_N + 1] (in t's allocation)
    int64_t blocks[FK_N][2] = {};     // block count of each kernel per shape
    int sms = 148;                    // the device's SM count (persistent network grid)
    WorkMap map(int k, int kind, int shape) const {
        return WorkMap{w0 + (((size_t)k * SK_N + kind) * 2 + shape) * (SK_N + 1), SK_N};
    }
};

// A system's own launch of kernel k over the slot of kind `kind` of its table, in the
// threads per block and register budget its launch configuration names.
Launch solo_launch(const Sys &s, int k, int kind);

}  // namespace sl
