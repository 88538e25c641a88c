// Line-kernel instantiations: float, FFT sizes n1 = 6 7 8 9 (0: Stockham).
#include "fcs_launch_impl.cuh"

FCS_INSTANTIATE_LINES(float, 6)
FCS_INSTANTIATE_LINES(float, 7)
FCS_INSTANTIATE_LINES(float, 8)
FCS_INSTANTIATE_LINES(float, 9)
