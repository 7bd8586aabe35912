// ops_2048.cu - kernels of the transform lengths 1536 and 2048 and of the
// grids 768 x 1536, 1024 x 2048 and their transposes (1024 x 2048 is the
// lateral grid of the paper's 10^6-PSF calculation).
#include "bpm_ops.cuh"

namespace bpmk {

void register_ops_2048(OpsRegistry& r) {
  add_length<1536, 0>(r);
  add_length<2048, 0>(r);
  add_grid<768, 1536>(r);
  add_grid<1536, 768>(r);
  add_grid<1024, 2048>(r);
  add_grid<2048, 1024>(r);
}

}  // namespace bpmk
