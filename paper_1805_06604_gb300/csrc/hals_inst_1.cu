// hals_inst_1.cu -- explicit instantiations of the HALS sweep kernel
// (hals_impl.cuh) for (lanes, slots) = (4, 31), (4, 18), (2, 20), (2, 10), (2, 3).
#include "hals_impl.cuh"

NMF_HALS_INSTANTIATE_ROWS(4, 31)
NMF_HALS_INSTANTIATE_ROWS(4, 18)
NMF_HALS_INSTANTIATE_ROWS(2, 20)
NMF_HALS_INSTANTIATE_ROWS(2, 10)
NMF_HALS_INSTANTIATE_ROWS(2, 3)
