// hals_inst_5.cu -- explicit instantiations of the HALS sweep kernel
// (hals_impl.cuh) for (lanes, slots) = (4, 27), (2, 31), (2, 24), (2, 14), (2, 5).
#include "hals_impl.cuh"

NMF_HALS_INSTANTIATE_ROWS(4, 27)
NMF_HALS_INSTANTIATE_ROWS(2, 31)
NMF_HALS_INSTANTIATE_ROWS(2, 24)
NMF_HALS_INSTANTIATE_ROWS(2, 14)
NMF_HALS_INSTANTIATE_ROWS(2, 5)
