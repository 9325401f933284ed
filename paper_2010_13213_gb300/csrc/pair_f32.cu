// pair_f32.cu -- pair-mode kernels instantiated for the float arithmetic.
#include "pair_ops.cuh"
template struct lgf::PairOps<float>;
