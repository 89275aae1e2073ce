// hals_inst_4.cu -- explicit instantiations of the HALS sweep kernel
// (hals_impl.cuh) for (lanes, slots) = (4, 20), (4, 13), (4, 10), (4, 8), (2, 8), (2, 2).
#include "hals_impl.cuh"

NMF_HALS_INSTANTIATE(4, 20)
NMF_HALS_INSTANTIATE(4, 13)
NMF_HALS_INSTANTIATE(4, 10)
NMF_HALS_INSTANTIATE(4, 8)
NMF_HALS_INSTANTIATE(2, 8)
NMF_HALS_INSTANTIATE(2, 2)
