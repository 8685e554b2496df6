// sl_rebuild.cuh -- argument blocks of the neighbour-list rebuild kernels (sl_neighbors.cu);
// a fused batch keeps one of each per replica slot (sl_batch.h).
#pragma once

#include "sl_internal.h"
#include "sl_fused.cuh"

namespace sl {

constexpr int LB_WARPS = 4;      // warps per block of the list build (one atom per warp)
constexpr int RB_THREADS = 256;  // threads per block of the binning kernels

struct GridArgs {
    int nc[3];
    double w[3];
    double inv2w[3];   // 2 / w: the half-width sub-cell index of x is floor(x * 2/w)
    int per[3];
};

// Every rebuild kernel's arguments for one system (binning, scan, scatter, finish).
struct BinArgs {
    const double4 *pos;
    const int32_t *species, *orig;
    int64_t n;
    GridArgs g;
    int ncell;
    int *count, *start, *fill, *atoms, *of;   // of: cell << 3 | sub-cell of each atom
    int *sub;              // [ncell][8] first position of each sub-cell, relative to its cell's start
    float4 *cposf;
    uint32_t *ckey;
    double4 *posref;
    unsigned long long *builds;
    int *rebuild;          // the system's rebuild flag (cleared after a conditional rebuild)
    const int *flag;       // null: unconditional; else the kernels return at once unless *flag
};

struct ListArgs {
    const double4 *pos;
    const int *cell_start, *cell_atoms, *cell_sub;
    const float4 *cposf;      // cell-ordered FP32 positions relative to each cell's corner, species and sub-cell bits in w
    int cap, cap_ang, capr;
    double cut_r2, cut_a2;
    float cut_r2f_lo, cut_r2f_hi, cut_a2f_lo, cut_a2f_hi;   // FP32 pre-test band
    float wf[3];              // cell widths in FP32 (the stencil cells' corner offsets)
    BoxDev<double> bd;
    BoxDev<float> bf;
    GridArgs g;
    int32_t *nbr;             // [n][capr] candidate lists, atom-major
    uint8_t *hash;            // [n][capr] 8-bit hash of each entry (index_hash8)
    int4 *seg;
    int *status;
    const int *flag;
};

struct RevArgs {
    const int32_t *species;
    const int32_t *nbr;   // atom-major [n][capr], capr a multiple of 32
    const uint8_t *hash;  // [n][capr] 8-bit hash of each entry (32-byte rows)
    const int4 *seg;
    int cap, capr;
    int64_t n;
    uint8_t *rev;         // [n][capr] reverse slots (cap <= 256)
    int *status;
    const int *flag;
};

// kernels of the group, in launch order (the flag is cleared after the last)
constexpr int RB_BIN = 0, RB_SCAN = 1, RB_SCATTER = 2, RB_CELLSORT = 3, RB_LISTS = 4, RB_REV = 5, RB_FINISH = 6,
              RB_KERNELS = 7;

struct RebuildPlan {
    BinArgs bin;
    ListArgs lists;
    RevArgs rev;
    int64_t blocks[RB_KERNELS];   // each kernel's block count for this system
};
RebuildPlan rebuild_plan(Sys &s, bool conditional);

}  // namespace sl
