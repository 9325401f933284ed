// box_df.cu -- block-index FFT mode instantiated for the df arithmetic.
#include "box_ops.cuh"
template struct lgf::BoxOps<df>;
