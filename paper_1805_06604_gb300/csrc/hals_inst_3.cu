// hals_inst_3.cu -- explicit instantiations of the HALS sweep kernel
// (hals_impl.cuh) for (lanes, slots) = (2, 32), (4, 11), (4, 9), (4, 6), (4, 4).
#include "hals_impl.cuh"

NMF_HALS_INSTANTIATE(2, 32)
NMF_HALS_INSTANTIATE(4, 11)
NMF_HALS_INSTANTIATE(4, 9)
NMF_HALS_INSTANTIATE(4, 6)
NMF_HALS_INSTANTIATE(4, 4)
