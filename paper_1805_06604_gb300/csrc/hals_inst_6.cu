// hals_inst_6.cu -- explicit instantiations of the HALS sweep kernel
// (hals_impl.cuh) for (lanes, slots) = (4, 26), (4, 20), (2, 25), (2, 15), (2, 7).
#include "hals_impl.cuh"

NMF_HALS_INSTANTIATE_ROWS(4, 26)
NMF_HALS_INSTANTIATE_ROWS(4, 20)
NMF_HALS_INSTANTIATE_ROWS(2, 25)
NMF_HALS_INSTANTIATE_ROWS(2, 15)
NMF_HALS_INSTANTIATE_ROWS(2, 7)
