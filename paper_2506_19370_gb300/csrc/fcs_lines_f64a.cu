// Line-kernel instantiations: double, FFT sizes n1 = 0 2 3 4 5 (0: Stockham).
#include "fcs_launch_impl.cuh"

FCS_INSTANTIATE_LINES(double, 0)
FCS_INSTANTIATE_LINES(double, 2)
FCS_INSTANTIATE_LINES(double, 3)
FCS_INSTANTIATE_LINES(double, 4)
FCS_INSTANTIATE_LINES(double, 5)
