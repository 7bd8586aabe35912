// ops_384.cu - kernels of the transform lengths 384 and 768 and of the grids
// 192 x 384, 384 x 768 and their transposes.
#include "bpm_ops.cuh"

namespace bpmk {

void register_ops_384(OpsRegistry& r) {
  add_length<384, 0>(r);
  add_length<768, 0>(r);
  add_grid<192, 384>(r);
  add_grid<384, 192>(r);
  add_grid<384, 768>(r);
  add_grid<768, 384>(r);
}

}  // namespace bpmk
