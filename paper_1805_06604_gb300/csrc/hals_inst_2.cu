// hals_inst_2.cu -- explicit instantiations of the HALS sweep kernel
// (hals_impl.cuh) for (lanes, slots) = (4, 24), (2, 15), (2, 11), (2, 7), (2, 4).
#include "hals_impl.cuh"

NMF_HALS_INSTANTIATE(4, 24)
NMF_HALS_INSTANTIATE(2, 15)
NMF_HALS_INSTANTIATE(2, 11)
NMF_HALS_INSTANTIATE(2, 7)
NMF_HALS_INSTANTIATE(2, 4)
