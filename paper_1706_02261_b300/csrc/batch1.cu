// batch1.cu - the batched kernel with schedule set 1: 256 as 4 x 8 x 8, 512 as unrolled 16 x 16 x 2, 1024 with four-step columns.
#include "batch.cuh"

namespace bpmk {

using BatchSched1 = BatchSched<1, 2, 0>;

BatchKernel batch_kernel_1() {
  BatchKernel k;
  k.fn = (const void*)bpm_batch_kernel<BatchSched1>;
  k.sched[0] = BatchSched1::s256;
  k.sched[1] = BatchSched1::s512;
  k.sched[2] = BatchSched1::s1024;
  return k;
}

}  // namespace bpmk
