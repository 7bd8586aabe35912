// batch0.cu - the batched kernel with schedule set 0: the default schedule of every size (256: 8 x 8 x 4, 512: the rolled radix-8 loop, 1024: four-step columns).
#include "batch.cuh"

namespace bpmk {

using BatchSched0 = BatchSched<0, 0, 0>;

BatchKernel batch_kernel_0() {
  BatchKernel k;
  k.fn = (const void*)bpm_batch_kernel<BatchSched0>;
  k.sched[0] = BatchSched0::s256;
  k.sched[1] = BatchSched0::s512;
  k.sched[2] = BatchSched0::s1024;
  return k;
}

}  // namespace bpmk
