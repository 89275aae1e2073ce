// hals_inst_8.cu -- explicit instantiations of the HALS sweep kernel
// (hals_impl.cuh) for (lanes, slots) = (4, 24), (4, 21), (4, 17), (2, 18).
#include "hals_impl.cuh"

NMF_HALS_INSTANTIATE_ROWS(4, 24)
NMF_HALS_INSTANTIATE_ROWS(4, 21)
NMF_HALS_INSTANTIATE_ROWS(4, 17)
NMF_HALS_INSTANTIATE_ROWS(2, 18)
