// hals_inst_9.cu -- explicit instantiations of the HALS sweep kernel
// (hals_impl.cuh) for (lanes, slots) = (4, 23), (4, 22), (2, 27), (2, 17).
#include "hals_impl.cuh"

NMF_HALS_INSTANTIATE_ROWS(4, 23)
NMF_HALS_INSTANTIATE_ROWS(4, 22)
NMF_HALS_INSTANTIATE_ROWS(2, 27)
NMF_HALS_INSTANTIATE_ROWS(2, 17)
