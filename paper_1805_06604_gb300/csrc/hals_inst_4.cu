// hals_inst_4.cu -- explicit instantiations of the HALS sweep kernel
// (hals_impl.cuh) for (lanes, slots) = (4, 28), (2, 30), (2, 23), (2, 13), (2, 8).
#include "hals_impl.cuh"

NMF_HALS_INSTANTIATE_ROWS(4, 28)
NMF_HALS_INSTANTIATE_ROWS(2, 30)
NMF_HALS_INSTANTIATE_ROWS(2, 23)
NMF_HALS_INSTANTIATE_ROWS(2, 13)
NMF_HALS_INSTANTIATE_ROWS(2, 8)
