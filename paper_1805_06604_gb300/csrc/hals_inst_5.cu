// hals_inst_5.cu -- explicit instantiations of the HALS sweep kernel
// (hals_impl.cuh) for (lanes, slots) = (2, 28), (4, 14), (2, 14), (2, 10), (4, 5), (2, 3).
#include "hals_impl.cuh"

NMF_HALS_INSTANTIATE(2, 28)
NMF_HALS_INSTANTIATE(4, 14)
NMF_HALS_INSTANTIATE(2, 14)
NMF_HALS_INSTANTIATE(2, 10)
NMF_HALS_INSTANTIATE(4, 5)
NMF_HALS_INSTANTIATE(2, 3)
