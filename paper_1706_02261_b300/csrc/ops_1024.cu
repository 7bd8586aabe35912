// ops_1024.cu - kernels of the transform length 1024 (two schedules) and of
// the 512 x 1024 and 1024 x 512 grids.
#include "bpm_ops.cuh"

namespace bpmk {

void register_ops_1024(OpsRegistry& r) {
  add_length<1024, 0>(r);
  add_length<1024, 1>(r);
  add_grid<512, 1024>(r);
  add_grid<1024, 512>(r);
}

}  // namespace bpmk
