// box_f32.cu -- block-index FFT mode instantiated for the float arithmetic.
#include "box_ops.cuh"
template struct lgf::BoxOps<float>;
