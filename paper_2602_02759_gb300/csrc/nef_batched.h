// nef_batched.h -- descriptors of the batched engine: many independent CP
// factorizations 'ir,jr,kr->ijk' (and random restarts of each) fitted together.
//
// Each (problem, restart) pair is a "unit".  The fit runs as one persistent
// launch per bond width whose CTAs take the units' fused passes from a device
// queue (PersistDesc below).  Work items of the restarts of one problem are
// adjacent, so the restarts read each Y tile from HBM once and from L2 after.
#pragma once

#include <cuda.h>

#include "nef_internal.h"

namespace nef {

constexpr int kMaxRestarts = 16;

// Finish of one unit in one mode phase (factor [rows x rank], S partials with
// rows padded and the bond padded to bp).
struct BatchFinish {
    float* theta;           // caller's factor, [rows x rank]
    float* canon32;         // canonical copy [rows_pad x bp]
    uint16_t* canon16;      // BF16 copy of the same layout
    const float* part_num;  // [n_split][rows_pad * bp]
    const float* part_den;
    int64_t rank, bp, s_size;
    int n_split;
    int64_t rows;           // rows of the factor (rows_pad = s_size / bp >= rows)
};

// Factor pointers of every restart of one problem (for the batched loss).
struct BatchFactors {
    const float* f[kMaxRestarts][3];
};

cudaError_t launch_pad_problem(const float* y, const uint8_t* mask, const int64_t* dims, const int64_t* pdims,
                               float* yp, uint32_t* bits, cudaStream_t st);

cudaError_t launch_mirror_batched(const BatchFinish* fin, const int64_t* prefix, int n_units, int64_t total,
                                  cudaStream_t st);

cudaError_t launch_loss_batched(const float* y, const uint8_t* mask, const int64_t* dims, int rank, int restarts,
                                const BatchFactors& fac, const LossSpec& L, double* part, int n_blocks,
                                double* out, cudaStream_t st);

// ---------------------------------------------------- batched tensor-core pass
struct TcUnitParams;  // defined with the kernel (k_view_tc.cuh)

// One unit of a batched launch: tensor maps of its padded Y view and of its
// TMA-staged column operands (consecutive rows, constant row), and the kernel
// parameters of its view pass.
struct alignas(64) TcUnit {
    CUtensorMap ymap;
    CUtensorMap vmap;
    CUtensorMap cmap;
    unsigned char prm[1152];  // tc::Params, copied byte-wise (size checked at compile time)
};

// Fill `unit` for view `v` (same rules as launch_view_tc); returns false if the
// view cannot run on the tensor cores.
bool tc_make_unit(const float* y, const uint32_t* mbits, const ViewDesc& v, const WeightSpec& w, int n_split,
                  float* s_num, float* s_den, int* err_flag, TcUnit* unit, int* n_rb);

// ------------------------------------------- persistent form: the whole fit, one launch
// A work item: the fused pass of (row block, column split) of one unit in one
// mode; items of one sweep are listed mode-major (all units' mode-0 items first).
struct PersistItem {
    int um;   // mode * n_units + unit: index of its TcUnit and BatchFinish
    int rb, sp;
    int pad;
};

struct PersistDesc {
    const TcUnit* units;          // [3 * n_units]
    const BatchFinish* fin;       // [3 * n_units]
    const PersistItem* items;     // [n_items]: one sweep
    const int* stage_items;       // [3 * n_units]: items of (mode, unit)
    const int* sweep_items;       // [n_units]: items of one sweep of the unit
    const int* prefix_items;      // [3 * n_units]: items of the unit's modes before this one
    int n_items, n_sweeps, n_units;
    int sweep0;                   // sweeps before this launch (its items are sweeps sweep0..)
    int bp;                       // bond_pad of every unit of the launch (16 or 32)
    unsigned int* queue;          // next item (0 at launch)
    unsigned int* done;           // [n_units] items of the unit completed (0 at launch)
    unsigned int* stage;          // [n_units] stages finished, mode by mode over the sweeps (0 at launch)
    int* err;                     // device error flag (bounded wait ran out)
    int* abort;                   // set with err: every CTA stops taking items
    UpdateSpec u;
    long long wait_cycles;        // limit of a wait for a preceding stage
};

// The fit of the units of one bond width as one launch of one CTA per SM: each CTA
// takes the next item of the queue, waits (bounded) until the unit's preceding
// stage has been updated, runs the fused pass, and the CTA completing a stage's
// last item applies that stage's update (split reduction, Eq. 3.4, operand copies).
cudaError_t launch_batched_persistent(const PersistDesc& d, const WeightSpec& w, int n_sm, cudaStream_t st);

}  // namespace nef
