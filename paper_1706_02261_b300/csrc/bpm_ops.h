// bpm_ops.h - the host side's view of the compiled kernels.
//
// The templated kernels (bpm_kernels.cuh) are instantiated in several
// translation units, one per group of transform lengths, which compile in
// parallel.  Each unit describes what it built in LenOps records (the
// half-step kernels of one transform length and schedule) and PairOps
// records (the persistent kernel of one grid), and bpm.cu finds them here.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "bpm_args.cuh"

namespace bpmk {

// The half-step kernels of one transform length n and schedule: rows of
// length n (ROW_* modes), columns of length n (COL_* modes), the light sheet.
struct LenOps {
  int n = 0, sched = 0;
  int schedules = 1;              // schedules of this length (0 .. schedules - 1)
  int is_default = 0;             // the schedule a single-field plan starts with
  int T = 0, NG = 0;              // threads per row or column, groups per CTA
  int four_step = 0;              // columns of this length use the four-step register layout
  int tw_count = 0;               // twiddles: forward, inverse, four-step tables
  size_t smem = 0;                // dynamic shared memory of the row / column kernels
  size_t line_smem = 0;           // ... of the light-sheet kernel
  // radix schedule, for tables built on the device (allocation-free entry)
  int loop = 0, loop_radix = 0, loop_passes = 0;     // rolled loop: one radix, paired table
  int nf = 0, rf[4] = {}, ni = 0, ri[4] = {};        // unrolled: forward / inverse radix lists
  cudaError_t (*init)(size_t smem_row_col, size_t smem_line) = nullptr;
  void (*twiddles)(std::vector<float2>& out) = nullptr;
  cudaError_t (*row)(int mode, bool kappa, int grid, const StepArgs& a, int z, cudaStream_t s) = nullptr;
  cudaError_t (*col)(int mode, int grid, const StepArgs& a, int z, cudaStream_t s) = nullptr;
  cudaError_t (*light_sheet)(int grid, const StepArgs& a, double w0, double xc, cudaStream_t s) = nullptr;
};

// The persistent kernel of one grid: rows of length nx, columns of length ny,
// in schedule `sched` (square grids) or the default schedules of the two
// lengths (rectangular grids: row_sched, col_sched).
struct PairOps {
  int nx = 0, ny = 0, sched = 0;
  int row_sched = 0, col_sched = 0;
  int row_ng = 0, col_ng = 0;     // row / column groups per CTA round
  int four_step = 0;              // the columns use the four-step register layout
  int col_hs = 0;                 // row stride (float2) of the staged propagator columns
  int tw_count = 0;               // twiddles of the combined table (rows, then columns)
  size_t smem_base = 0;           // dynamic shared memory before the staging buffers
  const void* kernel[2] = {nullptr, nullptr};   // without / with absorption
  void (*twiddles)(std::vector<float2>& out) = nullptr;
};

// registry of everything compiled (filled once, on first use)
const LenOps* find_len_ops(int n, int sched);
const PairOps* find_pair_ops(int nx, int ny, int sched);
const std::vector<int>& supported_lengths();

// the batched kernel in one schedule set (batch0.cu .. batch2.cu): the
// kernel and the schedules of the 256, 512 and 1024 transforms it uses
struct BatchKernel {
  const void* fn = nullptr;
  int sched[3] = {0, 0, 0};
  int sched_of(int n) const { return n == 256 ? sched[0] : (n == 512 ? sched[1] : (n == 1024 ? sched[2] : 0)); }
};
constexpr int kBatchKernels = 3;
BatchKernel batch_kernel_0();
BatchKernel batch_kernel_1();
BatchKernel batch_kernel_2();

// one call per translation unit of kernels (bpm.cu calls them all)
struct OpsRegistry {
  std::vector<LenOps> lens;
  std::vector<PairOps> pairs;
};
void register_ops_small(OpsRegistry& r);
void register_ops_256(OpsRegistry& r);
void register_ops_384(OpsRegistry& r);
void register_ops_512(OpsRegistry& r);
void register_ops_1024(OpsRegistry& r);
void register_ops_2048(OpsRegistry& r);

}  // namespace bpmk
