// nef_batched.h -- descriptors of the batched engine: many independent CP
// factorizations 'ir,jr,kr->ijk' (and random restarts of each) fitted together.
//
// Each (problem, restart) pair is a "unit".  A sweep runs three mode phases;
// in each phase one tensor-core launch covers every unit's fused pass (a CTA
// reads its unit and tile range from a work table), then one launch finishes
// every unit's factor update.  Work items of the restarts of one problem are
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
};

// Factor pointers of every restart of one problem (for the batched loss).
struct BatchFactors {
    const float* f[kMaxRestarts][3];
};

cudaError_t launch_pad_problem(const float* y, const uint8_t* mask, const int64_t* dims, const int64_t* pdims,
                               float* yp, uint32_t* bits, cudaStream_t st);

cudaError_t launch_finish_batched(const BatchFinish* fin, const int64_t* prefix, int n_units, int64_t total,
                                  const UpdateSpec& u, cudaStream_t st);

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

struct TcWork {
    int unit;
    int rb;   // row block
    int sp;   // column split
    int pad;
};

// Fill `unit` for view `v` (same rules as launch_view_tc); returns false if the
// view cannot run on the tensor cores.
bool tc_make_unit(const float* y, const uint32_t* mbits, const ViewDesc& v, const WeightSpec& w, int n_split,
                  float* s_num, float* s_den, int* err_flag, TcUnit* unit, int* n_rb);

// One launch over `n_work` work items of units that share bond_pad `bp`,
// weight kind and denominator mode.
cudaError_t launch_view_tc_batched(const TcUnit* units, const TcWork* work, int n_work, int bp, int need_den,
                                   const WeightSpec& w, cudaStream_t st);

}  // namespace nef
