// FP32 instantiation of the kernels (state and stencil arithmetic in FP32,
// FMA contraction allowed; the dt rule and all reductions stay FP64).
#include "kernels_impl.cuh"

namespace cm {

template struct Launch<float>;

}  // namespace cm
