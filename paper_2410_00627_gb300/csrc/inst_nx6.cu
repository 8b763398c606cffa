// Instantiates the device path for nx = 6 (one translation unit per state
// size so that the units compile in parallel).
#include "kernels.cuh"
SRTM_INSTANTIATE(6)
