// sl_batch.cu -- argument tables of the step kernels (sl_batch.h): their layout, a batch's
// plan kernel and captured graphs (one launch of each kernel covers every replica), and each
// system's own table.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sl_batch.h"
#include "sl_rebuild.cuh"

namespace sl {

// The step's work maps from the slots' budgets: slot r takes part while left[r] > 0, adding
// its block count of kernel k to map k; every budget that took part is then counted down by
// one.  Warp k scans the slots of kernel k, 32 at a time.
__global__ void __launch_bounds__(32 * FK_N) k_fused_plan(const int64_t *__restrict__ blocks, int64_t *left,
                                                        int64_t *__restrict__ w0, int cap) {
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t *w = w0 + (size_t)k * (cap + 1);
    int64_t carry = 0;
    for (int base = 0; base < cap; base += 32) {
        const int r = base + lane;
        const int64_t v = (r < cap && left[r] > 0) ? blocks[(size_t)k * cap + r] : 0;
        int64_t x = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (r < cap) w[r] = carry + x - v;
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) w[cap] = carry;
    __syncthreads();
    for (int r = threadIdx.x; r < cap; r += blockDim.x)
        if (left[r] > 0) left[r] -= 1;
}

void launch_fused_plan(const FusedTables &t, cudaStream_t st) {
    k_fused_plan<<<1, 32 * FK_N, 0, st>>>(t.at<int64_t>(t.o_blocks), reinterpret_cast<int64_t *>(t.dev + t.o_left),
                                          reinterpret_cast<int64_t *>(t.dev + t.o_w0), t.cap);
}

// atoms-per-block class of each kernel that takes one work item per block (-1: a loop over a
// work map: the rebuild group, and the tensor-core network)
static int item_class(int k, int prec) {
    switch (k) {
        case FK_FIRST: case FK_SECOND: return IC_HALF;
        case FK_CRAD: return IC_ATOM;
        case FK_ANG: case FK_BWD: return IC_QUAD;
        case FK_NET: return prec == 0 ? IC_ATOM : -1;
        default: return -1;
    }
}

// One step of every slot with a budget left, the default launch shapes: the one-item-per-block
// kernels over the block -> slot layout (a block whose slot takes no part returns at once), the
// others over the step's work maps with persistent grids.
void FusedBatch::enqueue(cudaStream_t st) const {
    auto L = [&](int k) {
        Launch x;
        x.m = t.map(k);
        const int c = item_class(k, t.prec);
        if (c >= 0) {
            x.item_slot = items + item_off[c];
            x.start = starts + (size_t)c * t.cap;
            x.grid = (unsigned)std::max<int64_t>(grid_items[c], 1);
        } else {
            x.grid = t.grid[k];
        }
        return x;
    };
    launch_fused_plan(t, st);
    launch_first_half_t(t, L(FK_FIRST), st);
    Launch rb[FK_FINISH - FK_BIN + 1];
    for (int k = FK_BIN; k <= FK_FINISH; ++k) rb[k - FK_BIN] = L(k);
    launch_rebuild_t(t, rb, true, true, st);
    const Launch ev[4] = {L(FK_CRAD), L(FK_ANG), L(FK_NET), L(FK_BWD)};
    if (t.prec == 0) launch_eval_t<double>(t, pd, ev, st, nullptr);
    else launch_eval_t<float>(t, pf, ev, st, nullptr);
    launch_second_half_t(t, L(FK_SECOND), true, st);
}

namespace {
size_t align_up(size_t x) { return (x + 127) & ~(size_t)127; }
}  // namespace

void fused_layout(FusedTables &t, int prec, int cap) {
    t.prec = prec;
    t.cap = cap;
    size_t first = 0, second = 0;
    fused_half_sizes(prec, &first, &second);
    size_t o = 0;
    auto take = [&](size_t &off, size_t bytes) {
        off = o;
        o = align_up(o + bytes);
    };
    take(t.o_blocks, sizeof(int64_t) * FK_N * cap);
    take(t.o_left, sizeof(int64_t) * cap);
    take(t.o_first, first * cap);
    take(t.o_second, second * cap);
    take(t.o_bin, sizeof(BinArgs) * cap);
    take(t.o_lists, sizeof(ListArgs) * cap);
    take(t.o_rev, sizeof(RevArgs) * cap);
    take(t.o_eval, fused_eval_size(prec) * cap);
    take(t.o_net, fused_net_size(prec) * cap);
    t.upload_bytes = o;
    take(t.o_w0, sizeof(int64_t) * FK_N * (cap + 1));
    t.bytes = o;
}

FusedBatch::~FusedBatch() { release(); }

void FusedBatch::release_graphs() {
    if (graph_g) cudaGraphExecDestroy(graph_g);
    if (graph_1) cudaGraphExecDestroy(graph_1);
    for (cudaGraph_t &x : tmpl) {
        if (x) cudaGraphDestroy(x);
        x = nullptr;
    }
    item_nodes.clear();
    graph_g = graph_1 = nullptr;
    g = 0;
}

void FusedBatch::release_items() {
    if (starts) cudaFree(starts);       // the allocation begins with the starts
    if (h_starts) cudaFreeHost(h_starts);
    items = nullptr;
    h_items = nullptr;
    starts = nullptr;
    h_starts = nullptr;
}

void FusedBatch::release() {
    release_graphs();
    release_items();
    if (t.dev) cudaFree(t.dev);
    if (img) cudaFreeHost(img);
    t = FusedTables();
    img = nullptr;
    dev_ = -1;
    atom_cap = 0;
    slot.clear();
    uid.clear();
    version.clear();
    stale.clear();
    have_model = false;
    follow = true;
    for (int64_t &x : grid_items) x = 0;
}

bool FusedBatch::setup(int prec, int cap, int device) {
    release();
    if (cap < 1 || cap > FUSED_MAX_SLOTS) return false;
    fused_layout(t, prec, cap);
    if (cudaMalloc((void **)&t.dev, t.bytes) != cudaSuccess) {
        t.dev = nullptr;
        release();
        return false;
    }
    if (cudaMallocHost((void **)&img, t.upload_bytes) != cudaSuccess) {
        img = nullptr;
        release();
        return false;
    }
    std::memset(img, 0, t.upload_bytes);
    if (cudaMemset(t.dev, 0, t.bytes) != cudaSuccess) {
        release();
        return false;
    }
    fused_grids_rebuild(t);   // persistent: the rebuild group and the tensor-core network
    fused_grid_net(t);
    dev_ = device;
    if (!reserve(1 << 16)) {
        release();
        return false;
    }
    slot.assign((size_t)cap, nullptr);
    uid.assign((size_t)cap, 0);
    version.assign((size_t)cap, 0);
    stale.assign((size_t)cap, 1);
    dirty = true;
    return true;
}

void FusedBatch::assign(int r, Sys *s) {
    if (r < 0 || r >= t.cap) return;
    // a system created after another was destroyed may sit at its address: compare ids
    if (uid[(size_t)r] != (s ? s->uid : 0)) stale[(size_t)r] = 1;
    slot[(size_t)r] = s;
}

bool FusedBatch::same_model(const Sys &s) const {
    return have_model && std::memcmp(&s.pd, &pd, sizeof pd) == 0 && std::memcmp(&s.pf, &pf, sizeof pf) == 0;
}

// The one-item-per-block class of a kernel of the step by its name (mangled: the identifier
// after its length; demangled: the identifier before its template or parameter list): the
// halves, the radial, angular and backward kernels and the FP64 network (the tensor-core
// network, k_mlp_tc, is persistent); -1 for the others.
static int item_kernel_class(const char *name) {
    struct { const char *id; int cls; } const k[] = {
        {"k_first_half", IC_HALF}, {"k_second_half", IC_HALF}, {"k_crad", IC_ATOM},
        {"k_mlp", IC_ATOM}, {"k_ang_fwd", IC_QUAD}, {"k_bwd", IC_QUAD}};
    for (const auto &x : k) {
        const std::string id(x.id);
        const std::string forms[3] = {std::to_string(id.size()) + id + "I", id + "<", id + "("};
        for (const std::string &f : forms)
            if (std::strstr(name, f.c_str())) return x.cls;
    }
    return -1;
}

bool FusedBatch::find_item_nodes(cudaGraph_t graph, cudaGraphExec_t exec, int steps) {
    size_t cnt = 0;
    if (cudaGraphGetNodes(graph, nullptr, &cnt) != cudaSuccess) return false;
    std::vector<cudaGraphNode_t> nodes(cnt);
    if (cnt && cudaGraphGetNodes(graph, nodes.data(), &cnt) != cudaSuccess) return false;
    int64_t found = 0;
    for (cudaGraphNode_t node : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(node, &ty) != cudaSuccess) return false;
        if (ty != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams p;
        if (cudaGraphKernelNodeGetParams(node, &p) != cudaSuccess) return false;
        const char *name = nullptr;
        if (cudaFuncGetName(&name, p.func) != cudaSuccess || !name) return false;
        const int c = item_kernel_class(name);
        if (c < 0) continue;
        if ((int64_t)p.gridDim.x != std::max<int64_t>(grid_items[c], 1)) return false;
        item_nodes.push_back(ItemNode{exec, node, c});
        ++found;
    }
    // per step: the two halves, the radial kernel (and the FP64 network), angular, backward
    return found == (int64_t)steps * (t.prec == 0 ? 6 : 5);
}

bool FusedBatch::resize_item_nodes() {
    for (const ItemNode &x : item_nodes) {
        cudaKernelNodeParams p;
        if (cudaGraphKernelNodeGetParams(x.node, &p) != cudaSuccess) return false;
        p.gridDim.x = (unsigned)std::max<int64_t>(grid_items[x.cls], 1);
        if (cudaGraphExecKernelNodeSetParams(x.exec, x.node, &p) != cudaSuccess) return false;
    }
    return true;
}

bool FusedBatch::graphs(int steps, const Sys &m, cudaStream_t st) {
    if (graph_g && g == steps && same_model(m)) return true;
    release_graphs();
    pd = m.pd;
    pf = m.pf;
    have_model = true;
    for (int which = 0; which < 2; ++which) {
        const int n = which == 0 ? steps : 1;
        cudaGraph_t graph;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
        for (int k = 0; k < n; ++k) enqueue(st);
        if (cudaStreamEndCapture(st, &graph) != cudaSuccess) return false;
        tmpl[which] = graph;   // kept: its kernel nodes name the ones a new layout resizes
        cudaGraphExec_t &exec = which == 0 ? graph_g : graph_1;
        const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) {
            exec = nullptr;
            release_graphs();
            return false;
        }
        if (follow && !find_item_nodes(graph, exec, n)) {
            // the graphs' grids cannot follow the layout: capacity grids from now on (the
            // failed query's error is not left for the next launch check)
            cudaGetLastError();
            follow = false;
            for (int c = 0; c < IC_N; ++c) grid_items[c] = item_cap[c];
            release_graphs();
            return graphs(steps, m, st);
        }
    }
    g = steps;
    ++captures;
    return true;
}

bool FusedBatch::reserve(int64_t atoms) {
    if (atoms <= atom_cap) return true;
    int64_t c = 1;
    while (c < atoms) c <<= 1;
    const int q = default_quad_block(t.prec);
    const int64_t per[IC_N] = {256, 128, q / 4};
    int64_t cap_items[IC_N], total = 0;
    for (int k = 0; k < IC_N; ++k) {
        cap_items[k] = (c + per[k] - 1) / per[k] + t.cap;   // whole blocks, one partial block per slot
        if (cap_items[k] > INT32_MAX) return false;
        total += cap_items[k];
    }
    release_graphs();
    release_items();
    const size_t bytes = sizeof(int) * (size_t)total + sizeof(int64_t) * IC_N * (size_t)t.cap;
    // one allocation each side: the 8-byte slot starts first, then the 4-byte layouts (so every
    // start stays aligned)
    if (cudaMalloc((void **)&starts, bytes) != cudaSuccess) {
        starts = nullptr;
        return false;
    }
    if (cudaMallocHost((void **)&h_starts, bytes) != cudaSuccess) {
        h_starts = nullptr;
        release_items();
        return false;
    }
    items = reinterpret_cast<int *>(starts + IC_N * (size_t)t.cap);
    h_items = reinterpret_cast<int *>(h_starts + IC_N * (size_t)t.cap);
    int64_t off = 0;
    for (int k = 0; k < IC_N; ++k) {
        item_off[k] = off;
        item_cap[k] = cap_items[k];
        off += cap_items[k];
    }
    item_bytes = bytes;
    atom_cap = c;
    layout_dirty = true;
    return true;
}

cudaError_t FusedBatch::upload(const int64_t *left, cudaStream_t st) {
    // the pinned image is reused: the previous call's copies are done before it changes
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    int64_t *blocks = reinterpret_cast<int64_t *>(img + t.o_blocks);
    for (int r = 0; r < t.cap; ++r) {
        Sys *s = slot[(size_t)r];
        if (!stale[(size_t)r] && (!s || version[(size_t)r] == s->capture_version)) continue;
        int64_t b[FK_N] = {};
        if (s) {
            fused_put_half(*s, r, t, img, b);
            fused_put_rebuild(*s, r, SK_STEP, t, img, b);
            fused_put_eval(*s, r, SK_STEP, t, img, b);
            fused_put_net(*s, r, SK_STEP, t, img, b);
            version[(size_t)r] = s->capture_version;
        }
        uid[(size_t)r] = s ? s->uid : 0;
        for (int k = 0; k < FK_N; ++k) blocks[(size_t)k * t.cap + r] = b[k];
        stale[(size_t)r] = 0;
        dirty = true;
    }
    int64_t atoms = 0;
    for (int r = 0; r < t.cap; ++r)
        if (slot[(size_t)r]) atoms += slot[(size_t)r]->n;
    if (!reserve(atoms)) return cudaErrorMemoryAllocation;
    if (dirty || layout_dirty) {
        // block -> slot layout of the one-item-per-block kernels: every occupied slot's blocks in
        // slot order, then no slot (-1) up to the capacity
        const int kof[IC_N] = {FK_FIRST, FK_CRAD, FK_ANG};
        for (int c = 0; c < IC_N; ++c) {
            int *it = h_items + item_off[c];
            int64_t o = 0;
            for (int r = 0; r < t.cap; ++r) {
                const int64_t nb = slot[(size_t)r] ? blocks[(size_t)kof[c] * t.cap + r] : 0;
                h_starts[(size_t)c * t.cap + r] = o;
                for (int64_t b = 0; b < nb; ++b) it[o + b] = r;
                o += nb;
            }
            grid_items[c] = follow ? std::max<int64_t>(o, 1) : item_cap[c];
            for (; o < item_cap[c]; ++o) it[o] = -1;
        }
        e = cudaMemcpyAsync(starts, h_starts, item_bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
        layout_dirty = false;
        // the captured graphs launch the new layout's blocks (the resize affects only their
        // later launches); where that fails they are captured again at the next step
        if (graph_g && !resize_item_nodes()) {
            cudaGetLastError();
            release_graphs();
        }
    }
    std::memcpy(img + t.o_left, left, sizeof(int64_t) * t.cap);
    if (dirty) e = cudaMemcpyAsync(t.dev, img, t.upload_bytes, cudaMemcpyHostToDevice, st);
    else e = cudaMemcpyAsync(t.dev + t.o_left, img + t.o_left, sizeof(int64_t) * t.cap, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) dirty = false;
    return e;
}

// ---------------------------------------------------------------- a system's own table
int solo_refresh(Sys &s) {
    if (!s.solo) {
        s.solo = new (std::nothrow) SoloTables();
        if (!s.solo) return -1;
    }
    SoloTables &so = *s.solo;
    FusedTables &t = so.t;
    const size_t w0_bytes = sizeof(int64_t) * FK_N * SK_N * 2 * (SK_N + 1);
    if (!t.dev) {
        fused_layout(t, s.prec, SK_N);
        if (cudaMalloc((void **)&t.dev, t.bytes + w0_bytes) != cudaSuccess) {
            t.dev = nullptr;
            return -1;
        }
        so.w0 = reinterpret_cast<int64_t *>(t.dev + t.bytes);
    }
    std::vector<unsigned char> &img = so.host;
    img.assign(t.bytes + w0_bytes, 0);
    int64_t b[SK_N][FK_N] = {};
    for (int kind = 0; kind < SK_N; ++kind) {
        fused_put_half(s, kind, t, img.data(), b[kind]);
        fused_put_rebuild(s, kind, kind, t, img.data(), b[kind]);
        fused_put_eval(s, kind, kind, t, img.data(), b[kind]);
        fused_put_net(s, kind, kind, t, img.data(), b[kind]);
    }
    // shape 0: the default threads per block; shape 1: half of them (radial: one atom per
    // thread; angular and backward: four threads per atom)
    for (int k = 0; k < FK_N; ++k) so.blocks[k][0] = so.blocks[k][1] = b[SK_STEP][k];
    const int q = default_quad_block(s.prec);
    so.blocks[FK_CRAD][1] = (s.n + 63) / 64;
    so.blocks[FK_ANG][1] = so.blocks[FK_BWD][1] = (s.n + q / 8 - 1) / (q / 8);
    // work maps covering slot `kind` alone
    int64_t *w = reinterpret_cast<int64_t *>(img.data() + t.bytes);
    for (int k = 0; k < FK_N; ++k)
        for (int kind = 0; kind < SK_N; ++kind)
            for (int shape = 0; shape < 2; ++shape) {
                int64_t *m = w + (((size_t)k * SK_N + kind) * 2 + shape) * (SK_N + 1);
                for (int r = 0; r <= SK_N; ++r) m[r] = r > kind ? so.blocks[k][shape] : 0;
            }
    cudaDeviceGetAttribute(&so.sms, cudaDevAttrMultiProcessorCount, s.device);
    if (cudaMemcpyAsync(t.dev, img.data(), img.size(), cudaMemcpyHostToDevice, s.stream) != cudaSuccess) return -1;
    return cudaStreamSynchronize(s.stream) == cudaSuccess ? 0 : -1;
}

void solo_free(Sys &s) {
    if (!s.solo) return;
    if (s.solo->t.dev) cudaFree(s.solo->t.dev);
    delete s.solo;
    s.solo = nullptr;
}

Launch solo_launch(const Sys &s, int k, int kind) {
    const SoloTables &so = *s.solo;
    Launch L;
    int shape = 0;
    const int q = default_quad_block(s.prec);
    if (k == FK_CRAD) {
        L.block = s.cfg.crad_block;
        L.minb = s.cfg.crad_minb;
        shape = L.block == 128 ? 0 : 1;
    } else if (k == FK_ANG) {
        L.block = s.cfg.ang_block ? s.cfg.ang_block : q;
        L.minb = s.cfg.ang_minb;
        shape = L.block == q ? 0 : 1;
    } else if (k == FK_BWD) {
        L.block = s.cfg.bwd_block ? s.cfg.bwd_block : q;
        L.minb = s.cfg.bwd_minb;
        shape = L.block == q ? 0 : 1;
    }
    L.m = so.map(k, kind, shape);
    int64_t g = so.blocks[k][shape];
    if (k == FK_NET && s.prec != 0) g = std::min<int64_t>(g, (int64_t)so.sms * s.cfg.mlp_ctas_per_sm);   // persistent
    L.grid = (unsigned)std::max<int64_t>(g, 1);
    // the argument block of slot `kind` as the kernel parameter (all but the rebuild group)
    const FusedTables &t = so.t;
    size_t first = 0, second = 0;
    fused_half_sizes(s.prec, &first, &second);
    const unsigned char *h = so.host.data();
    switch (k) {
        case FK_FIRST: L.solo = h + t.o_first + kind * first; break;
        case FK_SECOND: L.solo = h + t.o_second + kind * second; break;
        case FK_CRAD: case FK_ANG: case FK_BWD: L.solo = h + t.o_eval + kind * fused_eval_size(s.prec); break;
        case FK_NET: L.solo = h + t.o_net + kind * fused_net_size(s.prec); break;
        default:   // the rebuild group: a conditional one returns at once on the system's flag
            if (kind != SK_FULL) L.quick = s.rebuild;
            break;
    }
    return L;
}

}  // namespace sl
