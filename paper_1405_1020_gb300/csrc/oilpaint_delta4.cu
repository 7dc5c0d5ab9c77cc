// oilpaint_delta4.cu -- the straight-line difference-histogram kernels with
// 4 output columns per thread (see oilpaint_deltak.cuh).
#include "oilpaint_deltak.cuh"

namespace opk {

DeltaKFn deltak_kernel_k4(uint32_t nt, int nb, int r) { return deltak_kernel<4>(nt, nb, r); }

}  // namespace opk
