// Line-kernel instantiations: float, FFT sizes n1 = 0 2 3 4 5 (0: Stockham).
#include "fcs_launch_impl.cuh"

FCS_INSTANTIATE_LINES(float, 0)
FCS_INSTANTIATE_LINES(float, 2)
FCS_INSTANTIATE_LINES(float, 3)
FCS_INSTANTIATE_LINES(float, 4)
FCS_INSTANTIATE_LINES(float, 5)
