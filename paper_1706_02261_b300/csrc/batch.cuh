// batch.cuh - the batched kernel: many square instances of any supported size
// up to 1024 propagated by thread-block-cluster teams in one persistent launch
// (see the batched section of bpm_kernels.cuh).  Every size's code lives in
// one instruction stream; the transform schedule of each size is a template
// argument (a schedule set), and each set is compiled in a translation unit of
// its own (batch0.cu, batch1.cu, batch2.cu) so that bpm_autotune can time the
// sets on a plan's instances.
#pragma once
#include "bpm_kernels.cuh"
#include "bpm_ops.h"

namespace bpmk {

// schedule sets: the schedule of the 256, 512 and 1024 transforms (the other
// sizes have one)
template <int S256, int S512, int S1024>
struct BatchSched {
  static constexpr int s256 = S256, s512 = S512, s1024 = S1024;
  static constexpr int of(int n) { return n == 256 ? S256 : (n == 512 ? S512 : (n == 1024 ? S1024 : 0)); }
};

template <class SS>
__global__ void __launch_bounds__(kThreads, 1) bpm_batch_kernel(BatchArgs b) {
  extern __shared__ float4 smem_f4[];
  float2* smem = reinterpret_cast<float2*>(smem_f4);
  const int CL = (int)cluster_size(), rank = (int)cluster_rank(), cid = (int)cluster_id();
  bool bad = false;
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) b.slots[b.slot_base + cid] = batch_take(b);
    cluster_sync_all();
    const int k = ld_volatile(b.slots + b.slot_base + cid);
    cluster_sync_all();     // every CTA has read the slot before the leader may overwrite it
    if (k >= b.n_inst) break;
    const InstArgs ia = b.inst[b.order[k]];
    switch (ia.n) {
      case 64: batch_instance<Cfg<64>>(ia, b, rank, CL, smem, bad); break;
      case 128: batch_instance<Cfg<128>>(ia, b, rank, CL, smem, bad); break;
      case 192: batch_instance<Cfg<192>>(ia, b, rank, CL, smem, bad); break;
      case 256: batch_instance<Cfg<256, SS::s256>>(ia, b, rank, CL, smem, bad); break;
      case 384: batch_instance<Cfg<384>>(ia, b, rank, CL, smem, bad); break;
      case 512: batch_instance<Cfg<512, SS::s512>>(ia, b, rank, CL, smem, bad); break;
      case 1024: batch_instance<Cfg<1024, SS::s1024>>(ia, b, rank, CL, smem, bad); break;
      default: break;
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(b.err, 0, kDevErrNan);
}


}  // namespace bpmk
