// oilpaint_delta8.cu -- the straight-line difference-histogram kernels with
// 8 output columns per thread (see oilpaint_deltak.cuh).
#include "oilpaint_deltak.cuh"

namespace opk {

DeltaKFn deltak_kernel_k8(uint32_t nt, int nb, int r) { return deltak_kernel<8>(nt, nb, r); }

}  // namespace opk
