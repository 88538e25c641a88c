// Line-kernel instantiations: double, FFT sizes n1 = 6 7 8 9 (0: Stockham).
#include "fcs_launch_impl.cuh"

FCS_INSTANTIATE_LINES(double, 6)
FCS_INSTANTIATE_LINES(double, 7)
FCS_INSTANTIATE_LINES(double, 8)
FCS_INSTANTIATE_LINES(double, 9)
