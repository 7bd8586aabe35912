// batch.cu - the batched kernel: many square instances of any supported size
// up to 1024 propagated by thread-block-cluster teams in one persistent launch
// (see the batched section of bpm_kernels.cuh).
#include "bpm_kernels.cuh"
#include "bpm_ops.h"

namespace bpmk {

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
      case 64: batch_instance<64>(ia, b.err, rank, CL, smem, bad); break;
      case 128: batch_instance<128>(ia, b.err, rank, CL, smem, bad); break;
      case 192: batch_instance<192>(ia, b.err, rank, CL, smem, bad); break;
      case 256: batch_instance<256>(ia, b.err, rank, CL, smem, bad); break;
      case 384: batch_instance<384>(ia, b.err, rank, CL, smem, bad); break;
      case 512: batch_instance<512>(ia, b.err, rank, CL, smem, bad); break;
      case 1024: batch_instance<1024>(ia, b.err, rank, CL, smem, bad); break;
      default: break;
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(b.err, 0, kDevErrNan);
}

const void* batch_kernel_fn() { return (const void*)bpm_batch_kernel; }

}  // namespace bpmk
