// hals_inst_6.cu -- explicit instantiations of the HALS sweep kernel
// (hals_impl.cuh) for (lanes, slots) = (2, 24), (2, 20), (2, 16), (2, 13), (2, 9), (2, 5).
#include "hals_impl.cuh"

NMF_HALS_INSTANTIATE(2, 24)
NMF_HALS_INSTANTIATE(2, 20)
NMF_HALS_INSTANTIATE(2, 16)
NMF_HALS_INSTANTIATE(2, 13)
NMF_HALS_INSTANTIATE(2, 9)
NMF_HALS_INSTANTIATE(2, 5)
