// pair_df.cu -- pair-mode kernels instantiated for the df arithmetic.
#include "pair_ops.cuh"
template struct lgf::PairOps<df>;
