"""GB300-native FC-SDNN Runge-Kutta stage: C-ABI CUDA library and Python binding."""
