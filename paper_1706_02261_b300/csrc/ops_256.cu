// ops_256.cu - kernels of the transform length 256 (three schedules) and of
// the 128 x 256 and 256 x 128 grids.
#include "bpm_ops.cuh"

namespace bpmk {

void register_ops_256(OpsRegistry& r) {
  add_length<256, 0>(r);
  add_length<256, 1>(r);
  add_length<256, 2>(r);
  add_grid<128, 256>(r);
  add_grid<256, 128>(r);
}

}  // namespace bpmk
