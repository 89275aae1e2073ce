// hals_inst_2.cu -- explicit instantiations of the HALS sweep kernel
// (hals_impl.cuh) for (lanes, slots) = (4, 30), (2, 29), (2, 21), (2, 11), (2, 4).
#include "hals_impl.cuh"

NMF_HALS_INSTANTIATE_ROWS(4, 30)
NMF_HALS_INSTANTIATE_ROWS(2, 29)
NMF_HALS_INSTANTIATE_ROWS(2, 21)
NMF_HALS_INSTANTIATE_ROWS(2, 11)
NMF_HALS_INSTANTIATE_ROWS(2, 4)
