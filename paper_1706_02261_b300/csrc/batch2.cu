// batch2.cu - the batched kernel with schedule set 2: 256 as the rolled radix-16 loop, 512 as unrolled 8 x 8 x 8, 1024 with columns staged through shared memory.
#include "batch.cuh"

namespace bpmk {

using BatchSched2 = BatchSched<2, 1, 1>;

BatchKernel batch_kernel_2() {
  BatchKernel k;
  k.fn = (const void*)bpm_batch_kernel<BatchSched2>;
  k.sched[0] = BatchSched2::s256;
  k.sched[1] = BatchSched2::s512;
  k.sched[2] = BatchSched2::s1024;
  return k;
}

}  // namespace bpmk
