// hals_inst_7.cu -- explicit instantiations of the HALS sweep kernel
// (hals_impl.cuh) for (lanes, slots) = (4, 16), (4, 15), (4, 12), (2, 12), (4, 7), (4, 3).
#include "hals_impl.cuh"

NMF_HALS_INSTANTIATE(4, 16)
NMF_HALS_INSTANTIATE(4, 15)
NMF_HALS_INSTANTIATE(4, 12)
NMF_HALS_INSTANTIATE(2, 12)
NMF_HALS_INSTANTIATE(4, 7)
NMF_HALS_INSTANTIATE(4, 3)
