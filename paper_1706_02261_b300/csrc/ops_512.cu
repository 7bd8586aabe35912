// ops_512.cu - kernels of the transform length 512 (three schedules) and of
// the 256 x 512 and 512 x 256 grids.
#include "bpm_ops.cuh"

namespace bpmk {

void register_ops_512(OpsRegistry& r) {
  add_length<512, 0>(r);
  add_length<512, 1>(r);
  add_length<512, 2>(r);
  add_grid<256, 512>(r);
  add_grid<512, 256>(r);
}

}  // namespace bpmk
