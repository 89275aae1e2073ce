// hals_inst_0.cu -- explicit instantiations of the HALS sweep kernel
// (hals_impl.cuh) for (lanes, slots) = (4, 32).
#include "hals_impl.cuh"

NMF_HALS_INSTANTIATE(4, 32)
