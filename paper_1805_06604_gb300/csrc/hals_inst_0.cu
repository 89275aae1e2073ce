// hals_inst_0.cu -- explicit instantiations of the HALS sweep kernel
// (hals_impl.cuh) for (lanes, slots) = (4, 32), (2, 28), (2, 19), (2, 9).
#include "hals_impl.cuh"

NMF_HALS_INSTANTIATE_ROWS(4, 32)
NMF_HALS_INSTANTIATE_ROWS(2, 28)
NMF_HALS_INSTANTIATE_ROWS(2, 19)
NMF_HALS_INSTANTIATE_ROWS(2, 9)
