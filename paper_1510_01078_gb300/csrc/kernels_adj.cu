// Transposed NEDNER kernels (R^T and the sensor-position gradient).
#include <cuda_runtime.h>

#include "fft.cuh"
#include "internal.h"
