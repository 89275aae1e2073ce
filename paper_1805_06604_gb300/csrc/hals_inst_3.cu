// hals_inst_3.cu -- explicit instantiations of the HALS sweep kernel
// (hals_impl.cuh) for (lanes, slots) = (4, 29), (4, 19), (2, 22), (2, 12), (2, 6).
#include "hals_impl.cuh"

NMF_HALS_INSTANTIATE_ROWS(4, 29)
NMF_HALS_INSTANTIATE_ROWS(4, 19)
NMF_HALS_INSTANTIATE_ROWS(2, 22)
NMF_HALS_INSTANTIATE_ROWS(2, 12)
NMF_HALS_INSTANTIATE_ROWS(2, 6)
