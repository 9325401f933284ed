// pair_f64.cu -- pair-mode kernels instantiated for the double arithmetic.
#include "pair_ops.cuh"
template struct lgf::PairOps<double>;
