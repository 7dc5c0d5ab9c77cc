// oilpaint_delta2.cu -- the straight-line difference-histogram kernels with
// 2 output columns per thread (see oilpaint_deltak.cuh).
#include "oilpaint_deltak.cuh"

namespace opk {

DeltaKFn deltak_kernel_k2(uint32_t nt, int nb, int r) { return deltak_kernel<2>(nt, nb, r); }

}  // namespace opk
