// Host entry to the library's covariance check (small.cuh psd_check), so that
// its classification can be tested on the CPU against eigenvalues.
#include "small.cuh"

extern "C" int psd_check_host(const double* a, int n) { return srtm::psd_check<8>(a, n) ? 1 : 0; }
