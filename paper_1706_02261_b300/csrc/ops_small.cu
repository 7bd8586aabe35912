// ops_small.cu - kernels of the transform lengths 64, 96, 128 and 192 and of
// the grids built from them (square, and sides differing by a factor of two).
#include "bpm_ops.cuh"

namespace bpmk {

void register_ops_small(OpsRegistry& r) {
  add_length<64, 0>(r);
  add_length<96, 0>(r);
  add_length<128, 0>(r);
  add_length<192, 0>(r);
  add_grid<64, 128>(r);
  add_grid<128, 64>(r);
  add_grid<96, 192>(r);
  add_grid<192, 96>(r);
}

}  // namespace bpmk
