// sl_mlp_tc.cu -- the per-atom network on the 5th-generation tensor cores (tcgen05 + TMEM).
//
// Network (arXiv 2606.14073, Section 5.2.3 "ANN"; one hidden tanh layer):
//   E_i  = sum_h w1_h tanh(z_ih) - b1,   z_ih = sum_v W0_hv (s_v q_iv) - b0_h
//   Fp_iv = s_v sum_h t_ih W0_hv,        t_ih = w1_h (1 - tanh^2 z_ih)
// computed for tiles of 128 atoms as two dense contractions over atoms:
//   GEMM1  Z[128 x 32] = Q~[128 x 80] . W0^T[80 x 32]   (66 descriptor entries, 30 units, padded)
//   GEMM2  G[128 x 80] = T [128 x 32] . W0  [32 x 80]
// Operands are FP16 in shared memory in the canonical no-swizzle K-major layout
// (8-row x 16-byte core matrices; K-adjacent ones contiguous); every FP32 value x
// is split into hi = fp16(x), lo = fp16(x - hi) and each GEMM accumulates
// hi.hi + hi.lo + lo.hi in FP32 in tensor memory, which keeps the network within
// ~1e-6 relative of FP32 arithmetic.  One thread issues the MMAs; completion is
// signalled through an mbarrier (tcgen05.commit); the 128 threads read their
// atom's row back with tcgen05.ld (TMEM lane = atom row).  Persistent CTAs loop
// over tiles; the weights are staged once per CTA; each tile's 66 x 128 descriptors arrive
// by one TMA tile load (cp.async.bulk.tensor) issued while the previous tile is in the
// tensor cores.  Every wait is bounded: on timeout the kernel raises ST_TIMEOUT, waits for
// its own loads and MMAs, frees its tensor memory and returns.
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

#include "sl_internal.h"
#include "sl_batch.h"
#include "sl_fused.cuh"

namespace sl {
namespace tc {

constexpr int TM = 128;          // atoms per tile (MMA M)
constexpr int K1 = 80;           // descriptor entries padded to a multiple of 16
constexpr int N1 = 32;           // hidden units padded
constexpr int K2 = N1;
constexpr int N2 = K1;
constexpr int TMEM_COLS = 128;   // Z in columns [0, 32), G in [32, 112)

// shared memory (bytes)
constexpr uint32_t SZ_A1 = TM * K1 * 2;    // 20480
constexpr uint32_t SZ_B1 = N1 * K1 * 2;    // 5120
constexpr uint32_t SZ_A2 = TM * K2 * 2;    // 8192
constexpr uint32_t SZ_B2 = N2 * K2 * 2;    // 5120
constexpr uint32_t OFF_A1H = 0, OFF_A1L = OFF_A1H + SZ_A1;
constexpr uint32_t OFF_B1H = OFF_A1L + SZ_A1, OFF_B1L = OFF_B1H + SZ_B1;
// The A2 tile (layer-2 operand) reuses the A1 region: A1 is dead once the layer-1 MMAs
// have completed, and the next tile's A1 is written only after the layer-2 MMAs have.
// With the descriptor stage below, 95 KB per CTA: two CTAs share an SM.
constexpr uint32_t OFF_A2H = OFF_A1H, OFF_A2L = OFF_A2H + SZ_A2;
static_assert(2 * SZ_A2 <= SZ_A1, "A2 must fit in the A1 hi region");
constexpr uint32_t OFF_B2H = OFF_B1L + SZ_B1, OFF_B2L = OFF_B2H + SZ_B2;
// the four weight operands are one contiguous region, copied from a global image made once
constexpr uint32_t SZ_W = 2 * SZ_B1 + 2 * SZ_B2;         // 20480
static_assert(OFF_B1L == OFF_B1H + SZ_B1 && OFF_B2H == OFF_B1L + SZ_B1 && OFF_B2L == OFF_B2H + SZ_B2 &&
                  OFF_B1H % 16 == 0,
              "weight operands contiguous and 16-byte aligned");
constexpr uint32_t OFF_BAR = OFF_B2L + SZ_B2;            // 8-byte mbarrier: MMA completion
constexpr uint32_t OFF_BARQ = OFF_BAR + 8;                // 8-byte mbarrier: descriptor tile arrival
constexpr uint32_t OFF_TMEM = OFF_BARQ + 8;               // tensor-memory base address
// FP32 descriptors of the next tile, [DIM][TM] (the 66 x 128 box of the descriptor array),
// brought in by one TMA tile load while the current tile is in the tensor cores
constexpr uint32_t OFF_Q = (OFF_TMEM + 8 + 127) & ~127u;
constexpr uint32_t SZ_Q = DIM * TM * 4;                   // 33792, the TMA transaction size
constexpr uint32_t SMEM_BYTES = OFF_Q + SZ_Q;

// byte offset of element (row, k) of a [rows x K] 16-bit operand in the canonical
// no-swizzle K-major layout: core matrix = 8 rows x 8 elements (128 B, row stride 16 B),
// K-adjacent core matrices 128 B apart (LBO), 8-row groups K/8 * 128 B apart (SBO)
__host__ __device__ constexpr uint32_t cm_off(int row, int k, int K) {
    return (uint32_t)((row >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// tcgen05 shared-memory matrix descriptor: start address, LBO, SBO (all >> 4),
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor, kind::f16: D = F32, A = B = F16, both K-major, dense
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

constexpr int WAIT_LIMIT = 1 << 22;   // polls of a barrier before a wait gives up

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit = WAIT_LIMIT) {
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = __uint_as_float(r[t]);
}

// One TMA tile load of the descriptor box (atoms x0 .. x0+127, all 66 rows) into shared
// memory; its completion (SZ_Q bytes, zero-filled past the last atom) is counted on mbarrier
// `bar`, armed here with the expected byte count.  Issued by one thread.
__device__ __forceinline__ void tma_load_q(uint32_t dst, const CUtensorMap *map, int x0, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(SZ_Q) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x0), "r"(0), "r"(bar)
        : "memory");
}

// A tensor map read from global memory (the fused launch's replica table, written by a host
// copy): acquire it for the tensor-map proxy before the first copy through it.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// eight FP32 values -> 16 bytes of FP16 hi parts and 16 bytes of lo parts
__device__ __forceinline__ void split8(const float x[8], uint4 &hi, uint4 &lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const __half a = __float2half_rn(x[2 * t]), b = __float2half_rn(x[2 * t + 1]);
        const __half la = __float2half_rn(x[2 * t] - __half2float(a));
        const __half lb = __float2half_rn(x[2 * t + 1] - __half2float(b));
        h[t] = (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
        l[t] = (uint32_t)__half_as_ushort(la) | ((uint32_t)__half_as_ushort(lb) << 16);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// What a tile of the network needs: the descriptor map and first atom of its system, the
// system's atom count, outputs and status word.
struct MlpTile {
    const CUtensorMap *qmap;
    int x0;
    int64_t n;
    float *fp, *ei;
    int *status;
    bool gmem_map;   // the map lives in global memory (acquired before use)
};

// The weights' operand images: B1[h][v] = W0[h][v], B2[v][h] = W0[h][v] (zero padding), each
// FP32 value split into FP16 hi and lo, in the canonical layout at the byte offsets the tile
// kernel's shared memory uses (relative to OFF_B1H).  `dst` is shared or global memory.
__device__ __forceinline__ void weight_images(const NepDev<float> &P, unsigned char *dst, int tid, int nthreads) {
    for (int c = tid; c < N1 * (K1 / 8); c += nthreads) {      // B1: 32 rows x 10 chunks
        const int h = c / (K1 / 8), k0 = (c % (K1 / 8)) * 8;
        float x[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) x[t] = (h < NH && k0 + t < DIM) ? P.w0[h][k0 + t] : 0.f;
        uint4 hi, lo;
        split8(x, hi, lo);
        *reinterpret_cast<uint4 *>(dst + (OFF_B1H - OFF_B1H) + cm_off(h, k0, K1)) = hi;
        *reinterpret_cast<uint4 *>(dst + (OFF_B1L - OFF_B1H) + cm_off(h, k0, K1)) = lo;
    }
    for (int c = tid; c < N2 * (K2 / 8); c += nthreads) {      // B2: 80 rows x 4 chunks
        const int v = c / (K2 / 8), k0 = (c % (K2 / 8)) * 8;
        float x[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) x[t] = (v < DIM && k0 + t < NH) ? P.w0[k0 + t][v] : 0.f;
        uint4 hi, lo;
        split8(x, hi, lo);
        *reinterpret_cast<uint4 *>(dst + (OFF_B2H - OFF_B1H) + cm_off(v, k0, K2)) = hi;
        *reinterpret_cast<uint4 *>(dst + (OFF_B2L - OFF_B1H) + cm_off(v, k0, K2)) = lo;
    }
}

// the images of one model, made once per system
__global__ void __launch_bounds__(128) k_weight_images(const __grid_constant__ NepDev<float> P, unsigned char *img) {
    weight_images(P, img, threadIdx.x, blockDim.x);
}

// Body of the network kernel over the tiles src(0 .. total-1), each CTA taking tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...; wimg: the weights' operand images (global)
template <typename Src>
__device__ __forceinline__ void mlp_tc_body(const NepDev<float> &P, int64_t ntiles, const uint4 *__restrict__ wimg,
                                            Src src) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t bar = sbase + OFF_BAR, barq = sbase + OFF_BARQ;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + OFF_TMEM);

    // weights, once per CTA: a coalesced copy of the images (the same bytes the split of P.w0
    // gives, made once per system by k_weight_images)
    for (int k = tid; k < (int)(SZ_W / 16); k += blockDim.x)
        reinterpret_cast<uint4 *>(smem + OFF_B1H)[k] = __ldg(wimg + k);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(barq) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sbase + OFF_TMEM),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t t_z = tmem, t_g = tmem + N1;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;   // this warp's TMEM lane quadrant
    constexpr uint32_t IDESC1 = instr_desc(TM, N1), IDESC2 = instr_desc(TM, N2);
    uint32_t phase = 0, phase_q = 0;
    bool ok = true;
    bool q_in_flight = false;   // a descriptor tile load has been issued and not yet waited for
    int *status = nullptr;   // the status word of the last tile's system (timeouts are reported there)

    const float *stage = reinterpret_cast<const float *>(smem + OFF_Q);
    // the next tile's source, read while the current tile is in the tensor cores; thread 0
    // acquires each tensor map it has not used yet before the first copy through it
    const CUtensorMap *acquired = nullptr;
    auto issue = [&](const MlpTile &t) {
        if (t.gmem_map && t.qmap != acquired) {
            tensormap_acquire(t.qmap);
            acquired = t.qmap;
        }
        tma_load_q(sbase + OFF_Q, t.qmap, t.x0, barq);
    };
    MlpTile nxt;
    if (blockIdx.x < ntiles) {
        nxt = src(blockIdx.x);
        if (tid == 0) issue(nxt);
    }
    q_in_flight = blockIdx.x < ntiles;

    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const MlpTile cur = nxt;
        status = cur.status;
        const int64_t i = cur.x0 + tid;
        const bool valid = i < cur.n;
        float *__restrict__ fp = cur.fp;
        float *__restrict__ ei = cur.ei;
        const int64_t n = cur.n;
        // this tile's descriptors (every thread waits; the block agrees on the outcome)
        if (!__syncthreads_and(mbar_wait(barq, phase_q))) { ok = false; break; }
        phase_q ^= 1u;
        q_in_flight = false;
        // A1 row: s_v q_v, hi/lo
#pragma unroll
        for (int c = 0; c < K1 / 8; ++c) {
            float x[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int v = c * 8 + t;
                x[t] = v < DIM ? P.scal[v] * stage[v * TM + tid] : 0.f;
            }
            uint4 hi, lo;
            split8(x, hi, lo);
            *reinterpret_cast<uint4 *>(smem + OFF_A1H + cm_off(tid, c * 8, K1)) = hi;
            *reinterpret_cast<uint4 *>(smem + OFF_A1L + cm_off(tid, c * 8, K1)) = lo;
        }
        // every thread's reads of the stage are ordered before the next tile load, which
        // overlaps this tile's MMAs
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tile + gridDim.x < ntiles) {
            nxt = src(tile + gridDim.x);
            if (tid == 0) issue(nxt);
            q_in_flight = true;
        }
        if (tid == 0) {
            tc_fence_after();
            uint32_t acc = 0;
#pragma unroll
            for (int ks = 0; ks < K1 / 16; ++ks) {
                const uint32_t ko = ks * 256;
                const uint64_t ah = smem_desc(sbase + OFF_A1H + ko, 128, (K1 / 8) * 128);
                const uint64_t al = smem_desc(sbase + OFF_A1L + ko, 128, (K1 / 8) * 128);
                const uint64_t bh = smem_desc(sbase + OFF_B1H + ko, 128, (K1 / 8) * 128);
                const uint64_t bl = smem_desc(sbase + OFF_B1L + ko, 128, (K1 / 8) * 128);
                mma_f16(t_z, ah, bh, IDESC1, acc);
                acc = 1;
                mma_f16(t_z, ah, bl, IDESC1, 1);
                mma_f16(t_z, al, bh, IDESC1, 1);
            }
            mma_commit(bar);
        }
        // every thread waits; the block agrees on the outcome before anyone leaves the loop
        if (!__syncthreads_and(mbar_wait(bar, phase))) { ok = false; break; }
        phase ^= 1u;
        tc_fence_after();
        // epilogue 1: tanh layer, E_i, t_h into the A2 tile
        float z[N1];
        tmem_ld16(t_z + lane_off, z);
        tmem_ld16(t_z + lane_off + 16, z + 16);
        tmem_wait_ld();
        float tt[N1];
        float E = -P.b1;
#pragma unroll
        for (int h = 0; h < N1; ++h) {
            if (h < NH) {
                const float a = tanhf(z[h] - P.b0[h]);
                E += P.w1[h] * a;
                tt[h] = P.w1[h] * (1.f - a * a);
            } else {
                tt[h] = 0.f;
            }
        }
        if (valid) ei[i] = E;
#pragma unroll
        for (int c = 0; c < K2 / 8; ++c) {
            uint4 hi, lo;
            split8(tt + 8 * c, hi, lo);
            *reinterpret_cast<uint4 *>(smem + OFF_A2H + cm_off(tid, c * 8, K2)) = hi;
            *reinterpret_cast<uint4 *>(smem + OFF_A2L + cm_off(tid, c * 8, K2)) = lo;
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < K2 / 16; ++ks) {
                const uint32_t ko = ks * 256;
                const uint64_t ah = smem_desc(sbase + OFF_A2H + ko, 128, (K2 / 8) * 128);
                const uint64_t al = smem_desc(sbase + OFF_A2L + ko, 128, (K2 / 8) * 128);
                const uint64_t bh = smem_desc(sbase + OFF_B2H + ko, 128, (K2 / 8) * 128);
                const uint64_t bl = smem_desc(sbase + OFF_B2L + ko, 128, (K2 / 8) * 128);
                mma_f16(t_g, ah, bh, IDESC2, ks > 0 ? 1u : 0u);
                mma_f16(t_g, ah, bl, IDESC2, 1);
                mma_f16(t_g, al, bh, IDESC2, 1);
            }
            mma_commit(bar);
        }
        if (!__syncthreads_and(mbar_wait(bar, phase))) { ok = false; break; }
        phase ^= 1u;
        tc_fence_after();
        // epilogue 2: Fp_v = s_v G_v
#pragma unroll
        for (int c = 0; c < N2 / 16; ++c) {
            float g[16];
            tmem_ld16(t_g + lane_off + 16 * c, g);
            tmem_wait_ld();
            if (valid) {
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const int v = 16 * c + t;
                    if (v < DIM) fp[(int64_t)v * n + i] = P.scal[v] * g[t];
                }
            }
        }
        tc_fence_before();
        __syncthreads();   // TMEM and the A tiles are free for the next tile
    }
    if (!ok) {
        if (tid == 0 && status) atomicOr(status, ST_TIMEOUT);
        // let any MMA and any tile load still in flight finish before the memory is released
        // (bounded waits)
        mbar_wait(bar, phase);
        if (q_in_flight) mbar_wait(barq, phase_q);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// The network over the 128-atom tiles of a work map (sl_batch.h): a batch's (tab non-null;
// each slot's arguments and TMA map from the table, in global memory) or a system's own (tab
// null; its arguments, map included, as the kernel parameter solo).
__global__ void __launch_bounds__(128, 2) k_mlp_tc(const __grid_constant__ NepDev<float> P,
                                                   const MlpArgs *__restrict__ tab, WorkMap m,
                                                   const __grid_constant__ MlpArgs solo) {
    const int64_t total = __ldg(m.w0 + m.nrep);
    // the skip flag (the midpoint iteration's own launches only): uniform for the whole CTA and
    // before any shared-memory or TMEM use
    if (!tab && solo.skip && *solo.skip) return;
    // a CTA without a tile returns before any shared-memory or TMEM use (uniform)
    if ((int64_t)blockIdx.x >= total) return;
    // the slots taking part share the model: the weight images of the slot of this CTA's first tile
    const void *wimg = tab ? tab[work_replica(m, blockIdx.x)].wimg : solo.wimg;
    mlp_tc_body(P, total, reinterpret_cast<const uint4 *>(wimg), [&](int64_t g) {
        const int r = work_replica(m, g);
        const MlpArgs &a = tab ? tab[r] : solo;
        MlpTile t;
        t.qmap = &a.qmap;
        t.x0 = (int)((g - __ldg(m.w0 + r)) * TM);
        t.n = a.n;
        t.fp = a.fp;
        t.ei = a.ei;
        t.status = a.status;
        t.gmem_map = tab != nullptr;
        return t;
    });
}

// Self-test of the bounded wait: one thread waits on a barrier that nothing ever arrives
// at, gives up after `limit` polls and raises ST_TIMEOUT, as the network kernel does.
__global__ void k_selftest_wait(int limit, int *status) {
    __shared__ __align__(8) unsigned long long bar_storage;
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&bar_storage);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(bar, 0, limit)) atomicOr(status, ST_TIMEOUT);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

}  // namespace tc

int selftest_bounded_wait(int limit, int *status_out) {
    int *d;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return -1;
    cudaMemset(d, 0, sizeof(int));
    tc::k_selftest_wait<<<1, 1>>>(limit, d);
    cudaError_t e = cudaMemcpy(status_out, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? 0 : -1;
}

// TMA map of the FP32 descriptor array: a 2-D tensor of DIM rows x n atoms (atoms innermost,
// row stride qs * 4 bytes, a multiple of 16), read in boxes of 128 atoms x 66 rows; atoms past
// n read as zero.  The encode entry point is taken from the driver through the runtime.
int make_q_tensor_map(Sys &s) {
    if (s.prec == 0 || s.n == 0) return 0;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) != cudaSuccess ||
        qr != cudaDriverEntryPointSuccess || !fn)
        return -1;
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    const cuuint64_t dims[2] = {(cuuint64_t)s.n, (cuuint64_t)DIM};
    const cuuint64_t strides[1] = {(cuuint64_t)s.qs * 4};
    const cuuint32_t box[2] = {(cuuint32_t)tc::TM, (cuuint32_t)DIM};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = reinterpret_cast<Encode>(fn)(&s.qmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, s.q, dims, strides, box,
                                                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

// The network weights as the tensor-core kernel's operand images, made on the system's
// stream (ordered before its first evaluation) from its FP32 model parameters.
int make_mlp_image(Sys &s) {
    if (s.prec == 0 || s.n == 0) return 0;
    if (!s.mlp_img && cudaMalloc(&s.mlp_img, tc::SZ_W) != cudaSuccess) {
        s.mlp_img = nullptr;
        return -1;
    }
    tc::k_weight_images<<<1, 128, 0, s.stream>>>(s.pf, static_cast<unsigned char *>(s.mlp_img));
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---- argument tables (sl_batch.h): persistent CTAs over the slots' tiles
// the shared-memory limit is a per-device function attribute: set once per device
static void tc_smem_attribute(int dev) {
    static std::mutex mu;
    static uint64_t done = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (!(dev < 64 && (done >> dev & 1u))) {
        cudaFuncSetAttribute(tc::k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::SMEM_BYTES);
        if (dev < 64) done |= 1ull << dev;
    }
}

// the persistent grid of the tensor-core network (the FP64 network takes one work item per
// block: its grid follows the batch's atom capacity)
void fused_grid_net(FusedTables &t) {
    if (t.prec == 0) return;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    tc_smem_attribute(dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    t.grid[FK_NET] = (unsigned)(sms * LaunchCfg().mlp_ctas_per_sm);
}

void launch_net_t_tc(const FusedTables &t, const NepDev<float> &P, const Launch &L, cudaStream_t st) {
    int dev = 0;
    cudaGetDevice(&dev);
    tc_smem_attribute(dev);
    tc::k_mlp_tc<<<L.grid, 128, tc::SMEM_BYTES, st>>>(P, L.solo ? nullptr : t.at<MlpArgs>(t.o_net), L.m,
                                                       solo_args<MlpArgs>(L));
}

}  // namespace sl
