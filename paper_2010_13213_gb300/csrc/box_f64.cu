// box_f64.cu -- block-index FFT mode instantiated for the double arithmetic.
#include "box_ops.cuh"
template struct lgf::BoxOps<double>;
