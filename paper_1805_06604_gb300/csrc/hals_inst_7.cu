// hals_inst_7.cu -- explicit instantiations of the HALS sweep kernel
// (hals_impl.cuh) for (lanes, slots) = (4, 25), (2, 32), (2, 26), (2, 16), (2, 2).
#include "hals_impl.cuh"

NMF_HALS_INSTANTIATE_ROWS(4, 25)
NMF_HALS_INSTANTIATE_ROWS(2, 32)
NMF_HALS_INSTANTIATE_ROWS(2, 26)
NMF_HALS_INSTANTIATE_ROWS(2, 16)
NMF_HALS_INSTANTIATE_ROWS(2, 2)
