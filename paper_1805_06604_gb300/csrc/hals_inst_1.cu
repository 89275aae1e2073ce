// hals_inst_1.cu -- explicit instantiations of the HALS sweep kernel
// (hals_impl.cuh) for (lanes, slots) = (4, 28), (2, 6), (4, 2).
#include "hals_impl.cuh"

NMF_HALS_INSTANTIATE(4, 28)
NMF_HALS_INSTANTIATE(2, 6)
NMF_HALS_INSTANTIATE(4, 2)
